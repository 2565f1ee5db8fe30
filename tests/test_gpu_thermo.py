"""Thermally perfect gas (Sec. 2: specific heats from a NASA polynomial in
T) on the GPU against the oracle, through the C ABI.

States are built from primitive fields with the oracle's e(T), with a
temperature field spanning about 0.9 .. 1.6 so that gamma(T) varies by a
few percent across the box.  Tolerances are those of the calorically
perfect parity tests (the Newton inversions converge to rounding): one RHS
within 1e-13 of the flux scale, states after steps within 1e-11
field-normalised; mixed precision within its single-precision bars.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W
from tests.test_gpu_mixed import MIX_RHS_TOL, MIX_STEP_TOL
from tests.test_gpu_parity import RHS_TOL, STEP_TOL, field_err, flux_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A_TP = np.array([0.05, -0.2, 3.2, 0.5, -0.06, 0.004, 0.0])
A_CONST = np.array([0.0, 0.0, 1.4 / 0.4, 0.0, 0.0, 0.0, 0.0])


@pytest.fixture(scope="module")
def s2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import s2 as mod
    return mod


def hot_channel(nx, ny, nz, seed, a=A_TP):
    """The channel case's geometry and velocity field with a warm core:
    T = 1 + 0.6 (1 - y^2) (plus the case's perturbations through rho), walls
    at T_w = 1.  Returns the case and the state for the gas a."""
    c = W.channel(nx, ny, nz, seed=seed)
    rho = c.w0[0]
    u, v, w = c.w0[1] / rho, c.w0[2] / rho, c.w0[3] / rho
    Y = np.broadcast_to(c.y[None, :, None], rho.shape)
    T = 1.0 + 0.6 * (1.0 - Y ** 2)
    pr = problem(c, a)
    return c, pr, O.conserved(pr, rho, u, v, w, T)


def problem(c, a, **over):
    kw = dict(y=c.y, mach=c.mach, re=c.re, visc_exp=c.visc_exp, prandtl=c.prandtl, wall_y=c.wall_y,
              t_wall=c.t_wall, force=c.force, weno_order=c.weno_order, threshold=0.05, cp_coef=a)
    kw.update(over)
    return O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)


def solver(s2, pr, **kw):
    return s2.Solver(pr.nx, pr.ny, pr.nz, pr.lx, pr.ly, pr.lz, y=pr.y, mach=pr.mach, re=pr.re,
                     visc_exp=pr.visc_exp, prandtl=pr.prandtl, wall_y=pr.wall_y, t_wall=pr.t_wall,
                     force=pr.force, weno_order=pr.weno_order, threshold=pr.threshold,
                     cp_coeffs=pr.cp_coef, **kw)


def test_thermally_perfect_rhs_matches_oracle(s2):
    """One RHS of a walled, stretched, viscous, forced channel with WENO5 at
    part of the interfaces: flags identical, error within 1e-13 of the flux
    scale."""
    c, pr, w0 = hot_channel(40, 36, 24, seed=4)
    with solver(s2, pr, cfl=0.0, dt_fixed=1e-3) as sv:
        sv.set_state(w0)
        r = sv.rhs()
        f = sv.flags()
        st = sv.stats()
    assert st["status"] == 0
    ref, of = O.rhs(pr, w0, flags=True)
    frac = np.mean(np.concatenate([x.ravel() for x in of]))
    assert 0.01 < frac < 0.99, frac
    for a, b in zip(f, of):
        assert np.array_equal(a, b)
    S = np.maximum(flux_scale(w0, pr), np.max(np.abs(ref), axis=(1, 2, 3)))
    e = np.max(np.abs(r - ref), axis=(1, 2, 3)) / S
    print("thermally perfect rhs error / flux scale:", e, "weno fraction", frac)
    assert np.all(e < RHS_TOL), e


@pytest.mark.parametrize("weno,order", [(5, 6), (7, 8)])
def test_thermally_perfect_steps_match_oracle(s2, weno, order):
    """Ten RK3 steps at CFL 0.8 (dt from gamma(T) sound speeds), within
    1e-11 field-normalised: the walled channel with WENO5 / central 6, and
    a periodic box with WENO7 / central 8."""
    if weno == 5:
        c, pr, w0 = hot_channel(32, 28, 16, seed=6)
    else:
        n = 24
        pr = O.Problem(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi, mach=0.6, re=400.0, weno_order=7,
                       threshold=0.05, central_order=8, visc_order=8, cp_coef=A_TP)
        base = W.smooth_periodic(n, n, n, seed=9, mach=0.6, amp_u=0.8, amp_s=0.3)
        rho = base[0]
        u, v, w = base[1] / rho, base[2] / rho, base[3] / rho
        Z, Y, X = np.meshgrid(*(np.arange(n) * 2 * np.pi / n,) * 3, indexing="ij")
        T = 1.2 + 0.35 * np.sin(X) * np.cos(Y + Z)
        w0 = O.conserved(pr, rho, u, v, w, T)
    kw = dict(central_order=pr.central_order, visc_order=pr.visc_order)
    with solver(s2, pr, cfl=0.8, dt_every=3, **kw) as sv:
        sv.set_state(w0)
        sv.step(10)
        got = sv.get_state()
        st = sv.stats()
    ref, steps, dt = O.step(pr, w0, 10, cfl=0.8, dt_every=3)
    err = field_err(got, ref)
    print("thermally perfect state error after 10 steps:", err, "dt", dt)
    assert st["status"] == 0 and st["step"] == 10
    assert abs(st["dt"] - dt) < 1e-13 * dt
    assert np.all(err < STEP_TOL), err


def test_thermally_perfect_mixed_precision(s2):
    """Mixed precision (single-precision Newton inversion, flux and viscous
    arithmetic; double-precision state): one RHS against the oracle on the
    GPU's own flags, and ten steps."""
    c, pr, w0 = hot_channel(40, 36, 24, seed=4)
    with solver(s2, pr, precision="mixed", cfl=0.0, dt_fixed=1e-3) as sv:
        sv.set_state(w0)
        r = sv.rhs()
        f = sv.flags()
    ref = O.rhs_given_flags(pr, w0, f)
    S = np.maximum(flux_scale(w0, pr), np.max(np.abs(ref), axis=(1, 2, 3)))
    e = np.max(np.abs(r - ref), axis=(1, 2, 3)) / S
    print("mixed thermally perfect rhs error / flux scale:", e)
    assert np.all(e < MIX_RHS_TOL), e
    with solver(s2, pr, precision="mixed", cfl=0.8, dt_every=3) as sv:
        sv.set_state(w0)
        sv.step(10)
        got = sv.get_state()
    ref, _, _ = O.step(pr, w0, 10, cfl=0.8, dt_every=3)
    err = field_err(got, ref)
    print("mixed thermally perfect state error after 10 steps:", err)
    assert np.all(err < MIX_STEP_TOL), err


def test_constant_polynomial_matches_calorically_perfect_path(s2):
    """The thermally perfect kernels with c_p/R = gamma/(gamma-1) give the
    calorically perfect kernels' RHS to within 1e-13 of the flux scale."""
    c, pr, w0 = hot_channel(40, 36, 24, seed=4, a=A_CONST)
    prc = problem(c, None)
    out = []
    for p in (pr, prc):
        with solver(s2, p, cfl=0.0, dt_fixed=1e-3) as sv:
            sv.set_state(w0)
            out.append((sv.rhs(), sv.flags()))
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    S = np.maximum(flux_scale(w0, prc), np.max(np.abs(out[1][0]), axis=(1, 2, 3)))
    e = np.max(np.abs(out[0][0] - out[1][0]), axis=(1, 2, 3)) / S
    assert np.all(e < RHS_TOL), e


def test_thermally_perfect_noalloc_dt(s2):
    """s2_cfl_dt_noalloc with the thermally perfect gas gives the oracle's
    CFL dt."""
    import ctypes as C
    c, pr, w0 = hot_channel(32, 28, 16, seed=6)
    wd = torch.from_numpy(w0.reshape(-1)).cuda()
    ey = torch.from_numpy(O.metric(pr)[0]).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    grid = s2.s2_grid(pr.nx, pr.ny, pr.nz, pr.lx, pr.ly, pr.lz)
    cpc = np.ascontiguousarray(A_TP)
    gas = s2.s2_gas(pr.gamma, pr.prandtl, pr.mach, pr.re, pr.visc_exp, pr.t_ref)
    gas.cp_coeffs = cpc.ctypes.data_as(C.POINTER(C.c_double))
    P = C.c_void_p
    rc = s2._lib.s2_cfl_dt_noalloc(C.byref(grid), C.byref(gas), P(wd.data_ptr()), P(ey.data_ptr()), 0.8,
                                   P(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 0
    ref = O.dt(pr, w0, 0.8)
    assert abs(out.item() - ref) < 1e-13 * ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("gas", ["thermally_perfect", "calorically_perfect"])
def test_primitive_fields_round_trip(s2, gas, precision):
    """s2_set_primitives builds the oracle's conserved state from (rho, u,
    v, w, T) with E = e(T) + |u|^2/2, and s2_get_primitives recovers the
    fields, from host and from device buffers (the conversions are double
    precision in both modes)."""
    c = W.channel(24, 20, 12, seed=2)
    pr = problem(c, A_TP if gas == "thermally_perfect" else None)
    prim = c.prim0.copy()
    prim[4] = 1.0 + 0.6 * (1.0 - np.broadcast_to(c.y[None, :, None], prim[4].shape) ** 2)
    ref = O.conserved(pr, *prim)
    with solver(s2, pr, cfl=0.8, precision=precision) as sv:
        sv.set_primitives(prim)
        w_host = sv.get_state()
        back_host = sv.get_primitives()
        sv.set_primitives(torch.from_numpy(prim).cuda())
        w_dev = sv.get_state()
        back_dev = torch.zeros(prim.shape, dtype=torch.float64, device="cuda")
        sv.get_primitives(back_dev)
        back_dev = back_dev.cpu().numpy()
    for w in (w_host, w_dev):
        assert np.all(field_err(w, ref) < 1e-15), field_err(w, ref)
    for back in (back_host, back_dev):
        assert np.all(field_err(back, prim) < 1e-14), field_err(back, prim)


def test_batch_with_thermally_perfect_members_matches_solo_runs(s2):
    """Thermally perfect members (FP64 and mixed) stepped in one batch with
    a calorically perfect one give their solo results bit for bit."""
    c, pr, w0 = hot_channel(24, 20, 12, seed=8)
    _, prc, _ = hot_channel(24, 20, 12, seed=8, a=None)
    specs = [(pr, dict(precision="fp64")), (pr, dict(precision="mixed")), (prc, dict(precision="mixed"))]
    states = [w0, w0, c.w0]

    def run(batch):
        svs = []
        for (p, kw), w in zip(specs, states):
            sv = solver(s2, p, cfl=0.8, dt_every=2, **kw)
            sv.set_state(w)
            svs.append(sv)
        if batch:
            with s2.Batch(svs) as b:
                b.step(5)
                b.sync()
        else:
            for sv in svs:
                sv.step(5)
        out = [sv.get_state() for sv in svs]
        for sv in svs:
            sv.close()
        return out

    for a, b in zip(run(True), run(False)):
        assert np.array_equal(a, b)
