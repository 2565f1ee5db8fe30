"""Mixed precision (single-precision primitives, flux, WENO and viscous
arithmetic; double-precision state, RK accumulation and E -> T recovery)
against the FP64 oracle.

The sensor of the mixed path decides in single precision, so its flags can
differ from the oracle's at interfaces whose sensor is within rounding of the
threshold.  The arithmetic is therefore compared with the oracle evaluated
on the GPU's own flags (or_rhs_given_flags); the flag disagreement is counted
separately.  Errors are printed (the statement of each result) and bounded.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W
from tests.test_gpu_parity import case_kw, field_err, flux_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# single precision: 2^-24 = 6e-8 per operation; the flux divergence keeps
# it relative to the flux magnitude (measured <= 6e-7 of the flux scale).
# After 10 steps the field-normalised error is ~1e-7..1e-6, except for a
# field that starts at zero (rho w of the Taylor-Green vortex, whose
# maximum after 10 steps is ~1e-2 of the velocity scale): ~8e-5.
MIX_RHS_TOL = 2e-6
MIX_STEP_TOL = 3e-4


@pytest.fixture(scope="module")
def s2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import s2 as mod
    return mod


def mixed_rhs_err(s2, w0, dims, kw):
    nx, ny, nz, lx, ly, lz = dims
    pkw = {k: v for k, v in kw.items() if k not in ("cfl", "dt_fixed", "dt_every")}
    pr = O.Problem(nx, ny, nz, lx, ly, lz, **pkw)
    with s2.Solver(nx, ny, nz, lx, ly, lz, precision="mixed", cfl=0.0, dt_fixed=1e-3, **pkw) as sv:
        sv.set_state(w0)
        r = sv.rhs()
        f = sv.flags()
    ref_own, of = O.rhs(pr, w0, flags=True)
    ref = O.rhs_given_flags(pr, w0, f) if pr.weno_order else ref_own
    S = np.maximum(flux_scale(w0, pr), np.max(np.abs(ref), axis=(1, 2, 3)))
    e = np.max(np.abs(r - ref), axis=(1, 2, 3)) / S
    flips = sum(int(np.sum(a != b)) for a, b in zip(f, of))
    total = sum(a.size for a in f)
    print("mixed rhs error / flux scale:", e, "flag flips: %d of %d" % (flips, total))
    return e, flips, total


def test_mixed_rhs_tgv_and_channel(s2):
    c = W.taylor_green(32)
    e, _, _ = mixed_rhs_err(s2, c.w0, (c.nx, c.ny, c.nz, c.lx, c.ly, c.lz),
                            dict(mach=c.mach, re=c.re, weno_order=0))
    assert np.all(e < MIX_RHS_TOL), e
    ch = W.channel(64, 48, 32, seed=7)
    kw = case_kw(ch)
    kw["threshold"] = 0.05
    e, flips, total = mixed_rhs_err(s2, ch.w0, (ch.nx, ch.ny, ch.nz, ch.lx, ch.ly, ch.lz), kw)
    assert np.all(e < MIX_RHS_TOL), e
    assert flips <= 1e-3 * total


@pytest.mark.parametrize("weno", [0, 5])
def test_mixed_rhs_keep(s2, weno):
    """KEEP central flux (exact logarithmic means) in single precision
    against the FP64 oracle, central and hybrid."""
    nx, ny, nz = 37, 29, 19
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=81, mach=0.7, amp_u=0.7, amp_s=0.25)
    xi = np.arange(ny) * L / ny
    kw = dict(y=xi + 0.25 * np.sin(xi), mach=0.7, re=150.0, weno_order=weno, threshold=0.15, keep=-1)
    e, flips, total = mixed_rhs_err(s2, w0, (nx, ny, nz, L, L, L), kw)
    assert np.all(e < MIX_RHS_TOL), e
    assert flips <= 1e-3 * total


@pytest.mark.parametrize("weno", [5, 7])
def test_mixed_rhs_ragged_hybrid(s2, weno):
    nx, ny, nz = 37, 29, 19
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=48, mach=0.7, amp_u=0.7, amp_s=0.25)
    xi = np.arange(ny) * L / ny
    kw = dict(y=xi + 0.25 * np.sin(xi), mach=0.7, re=150.0, weno_order=weno, threshold=0.15)
    e, flips, total = mixed_rhs_err(s2, w0, (nx, ny, nz, L, L, L), kw)
    assert np.all(e < MIX_RHS_TOL), e
    assert flips <= 1e-3 * total


@pytest.mark.parametrize("case", ["tgv", "channel"])
def test_mixed_10_steps_against_fp64_oracle(s2, case):
    if case == "tgv":
        c = W.taylor_green(32)
    else:
        c = W.channel(64, 48, 32, seed=7)
    kw = case_kw(c)
    pr = O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)
    with s2.Solver.from_case(c, precision="mixed", cfl=0.8, dt_every=10) as sv:
        sv.set_state(c.w0)
        sv.step(10)
        w = sv.get_state()
        st = sv.stats()
    ref, _, dt = O.step(pr, c.w0, 10, cfl=0.8, dt_every=10)
    err = field_err(w, ref)
    print("%s mixed vs FP64 oracle after 10 steps (field-normalised):" % case, err,
          "dt rel diff %.2e" % abs(st["dt"] / dt - 1))
    assert np.all(np.isfinite(w))
    assert np.all(err < MIX_STEP_TOL), err


def test_mixed_conservation_periodic(s2):
    """Flux-form increments summed in double precision: the volume integrals
    of the conserved variables drift only by single-precision rounding."""
    nx, ny, nz = 40, 36, 32
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=9, mach=0.8, amp_u=0.7, amp_s=0.2)
    with s2.Solver(nx, ny, nz, L, L, L, mach=0.8, re=-1.0, weno_order=5, threshold=0.1, cfl=0.5, dt_every=1,
                   precision="mixed") as sv:
        sv.set_state(w0)
        s0 = sv.stats()
        sv.step(20)
        s1 = sv.stats()
    drift = {k: abs(s1[k] - s0[k]) / abs(s0[k]) for k in ("mass", "energy")}
    print("mixed conservation drift over 20 steps:", drift)
    assert drift["mass"] < 1e-6 and drift["energy"] < 1e-6


@pytest.mark.parametrize("orders", [(2, 2, 1), (2, 2, 3), (4, 4, 5), (8, 8, 7)])
def test_mixed_rhs_orders_walls_ragged(s2, orders):
    """Mixed path at other central / viscous / WENO orders on a channel
    whose sizes are not multiples of any tile (walls, stretched y,
    forcing): every stencil width of the single-precision kernels,
    including the divergence ghosts they write at the walls."""
    co, vo, wo = orders
    c = W.channel(45, 30, 21, seed=17)
    kw = case_kw(c)
    kw.update(central_order=co, visc_order=vo, weno_order=wo, threshold=0.05)
    e, flips, total = mixed_rhs_err(s2, c.w0, (c.nx, c.ny, c.nz, c.lx, c.ly, c.lz), kw)
    assert np.all(e < MIX_RHS_TOL), e
    assert flips <= 1e-3 * total
