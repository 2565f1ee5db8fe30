"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances.  States after 10 RK3 steps: max abs error per conserved field
over the field's max abs value below 1e-11 (the bar of the FP64 path).
One RHS evaluation: the flux divergence loses digits relative to the fluxes
it differences (at low Mach the pressure, ~1/(gamma M^2), is ~10^3 times
its gradient), so the error per field is measured against
S_f = max(max|R_f|, max_points sum_d |F_f,d| / h_d) with F the convective
flux (pressure included) and h_d the smallest spacing; the bar is 1e-13 of
S_f (about 450 ulp of the flux).  WENO flags must be identical.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHS_TOL = 1e-13
STEP_TOL = 1e-11


@pytest.fixture(scope="module")
def s2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import s2 as mod
    return mod


def field_err(a, b):
    scale = np.max(np.abs(b), axis=(1, 2, 3))
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(a - b), axis=(1, 2, 3)) / scale


def flux_scale(w, pr):
    """S_f of the module docstring for the state w of problem pr."""
    g = pr.gamma
    R = 1.0 / (g * pr.mach ** 2)
    rho = w[0]
    u = [w[1] / rho, w[2] / rho, w[3] / rho]
    q2 = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    T = (w[4] / rho - 0.5 * q2) * (g - 1.0) / R
    p = rho * R * T
    H = g / (g - 1.0) * R * T + 0.5 * q2
    ey, _ = O.metric(pr)
    inv_h = [pr.nx / pr.lx, float(np.max(ey)), pr.nz / pr.lz]
    S = np.zeros(5)
    acc = [np.zeros_like(rho) for _ in range(5)]
    for d in range(3):
        un = np.abs(rho * u[d])
        acc[0] += un * inv_h[d]
        for a in range(3):
            acc[1 + a] += (np.abs(rho * u[d] * u[a]) + (np.abs(p) if a == d else 0.0)) * inv_h[d]
        acc[4] += un * np.abs(H) * inv_h[d]
    for f in range(5):
        S[f] = np.max(acc[f])
    return S


def rhs_err(a, b, w, pr):
    S = np.maximum(flux_scale(w, pr), np.max(np.abs(b), axis=(1, 2, 3)))
    e = np.max(np.abs(a - b), axis=(1, 2, 3)) / S
    print("rhs error / flux scale:", e)
    return e


def make(s2, nx, ny, nz, lx, ly, lz, **kw):
    sk = dict(kw)
    ok = {k: v for k, v in kw.items() if k in ("y", "gamma", "prandtl", "mach", "re", "visc_exp", "t_ref",
                                               "wall_y", "t_wall", "force", "weno_order", "threshold",
                                               "central_order", "visc_order", "keep")}
    return s2.Solver(nx, ny, nz, lx, ly, lz, **sk), O.Problem(nx, ny, nz, lx, ly, lz, **ok)


def rhs_parity(s2, w0, nx, ny, nz, lx, ly, lz, **kw):
    sv, pr = make(s2, nx, ny, nz, lx, ly, lz, cfl=0.0, dt_fixed=1e-3, **kw)
    with sv:
        sv.set_state(w0)
        r = sv.rhs()
        f = sv.flags()
    ref, of = O.rhs(pr, w0, flags=True)
    return rhs_err(r, ref, w0, pr), f, of


def taylor_green_case():
    return W.taylor_green(32)


def test_tgv32_rhs_and_10_steps(s2):
    """Taylor-Green 32^3, central only, 10 steps at CFL 0.8."""
    c = taylor_green_case()
    kw = dict(mach=c.mach, re=c.re, visc_exp=c.visc_exp, prandtl=c.prandtl, weno_order=0)
    e, _, _ = rhs_parity(s2, c.w0, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)
    assert np.all(e < RHS_TOL), e
    sv, pr = make(s2, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cfl=0.8, dt_every=10, **kw)
    with sv:
        sv.set_state(c.w0)
        sv.step(10)
        w = sv.get_state()
        st = sv.stats()
    ref, steps, dt = O.step(pr, c.w0, 10, cfl=0.8, dt_every=10)
    err = field_err(w, ref)
    print("state error after 10 steps:", err)
    assert np.all(err < STEP_TOL), err
    assert st["step"] == 10 and abs(st["dt"] - dt) < 1e-14 * dt
    assert abs(st["t"] - 10 * dt) < 1e-12


def channel_small(nx=64, ny=48, nz=32, seed=7):
    return W.channel(nx, ny, nz, seed=seed)


def case_kw(c):
    return dict(y=c.y, mach=c.mach, re=c.re, visc_exp=c.visc_exp, prandtl=c.prandtl, wall_y=c.wall_y,
                t_wall=c.t_wall, force=c.force, weno_order=c.weno_order, threshold=c.threshold)


def test_channel_small_rhs_flags_and_10_steps(s2):
    """Channel with walls, tanh y, forcing, hybrid WENO5 (reduced grid)."""
    c = channel_small()
    kw = case_kw(c)
    kw["threshold"] = 0.05  # more flagged interfaces at this size
    e, f, of = rhs_parity(s2, c.w0, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)
    assert np.all(e < RHS_TOL), e
    for a, b in zip(f, of):
        assert np.array_equal(a, b)
    frac = np.mean(np.concatenate([a.ravel() for a in of]))
    assert 0.01 < frac < 0.9, frac
    sv, pr = make(s2, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cfl=0.8, dt_every=10, **kw)
    with sv:
        sv.set_state(c.w0)
        sv.step(10)
        w = sv.get_state()
    ref, _, _ = O.step(pr, c.w0, 10, cfl=0.8, dt_every=10)
    err = field_err(w, ref)
    assert np.all(err < STEP_TOL), err


@pytest.mark.parametrize("shape", [(37, 29, 19), (150, 70, 40), (1, 5, 3), (5, 1, 7)])
@pytest.mark.parametrize("weno", [0, 5, 7])
def test_ragged_sizes_stretched_hybrid(s2, shape, weno):
    """Sizes that are not multiples of any tile (and degenerate 1-point
    directions), periodic stretched y, viscous, hybrid WENO."""
    nx, ny, nz = shape
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=11 + nx, mach=0.7, amp_u=0.7, amp_s=0.25)
    xi = np.arange(ny) * L / ny
    y = xi + 0.25 * np.sin(xi) if ny > 1 else None
    kw = dict(y=y, mach=0.7, re=150.0, visc_exp=0.76, weno_order=weno, threshold=0.15)
    e, f, of = rhs_parity(s2, w0, nx, ny, nz, L, L, L, **kw)
    assert np.all(e < RHS_TOL), e
    if weno:
        for a, b in zip(f, of):
            assert np.array_equal(a, b)


def test_weno_everywhere_double_sod(s2):
    """WENO5 forced everywhere on the 1-D double Sod problem (ny = nz = 1)."""
    n = 200
    w0, x, mach = W.double_sod(n)
    kw = dict(mach=mach, re=-1.0, weno_order=5, threshold=-1.0)
    sv, pr = make(s2, n, 1, 1, 2.0, 1.0, 1.0, cfl=0.0, dt_fixed=1e-3, **kw)
    with sv:
        sv.set_state(w0)
        r = sv.rhs()
        sv.step(10)
        w = sv.get_state()
    ref = O.rhs(pr, w0)
    assert np.all(rhs_err(r, ref, w0, pr) < RHS_TOL)
    wr, _, _ = O.step(pr, w0, 10, dt_fixed=1e-3)
    assert np.all(field_err(w, wr) < STEP_TOL)


def test_weno7_periodic_box(s2):
    nx, ny, nz = 48, 40, 36
    w0 = W.smooth_periodic(nx, ny, nz, seed=5, mach=0.9, amp_u=0.8, amp_s=0.3)
    kw = dict(mach=0.9, re=400.0, weno_order=7, threshold=0.1)
    sv, pr = make(s2, nx, ny, nz, 2 * np.pi, 2 * np.pi, 2 * np.pi, cfl=0.6, dt_every=3, **kw)
    with sv:
        sv.set_state(w0)
        r = sv.rhs()
        sv.step(10)
        w = sv.get_state()
    assert np.all(rhs_err(r, O.rhs(pr, w0), w0, pr) < RHS_TOL)
    wr, _, _ = O.step(pr, w0, 10, cfl=0.6, dt_every=3)
    assert np.all(field_err(w, wr) < STEP_TOL)


def test_full_channel_rhs_and_steps(s2):
    """The benchmark's channel workload at full size, 256x128x128."""
    c = W.channel()
    kw = case_kw(c)
    e, f, of = rhs_parity(s2, c.w0, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)
    assert np.all(e < RHS_TOL), e
    for a, b in zip(f, of):
        assert np.array_equal(a, b)
    sv, pr = make(s2, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cfl=0.8, dt_every=10, **kw)
    with sv:
        sv.set_state(c.w0)
        sv.step(3)
        w = sv.get_state()
    ref, _, _ = O.step(pr, c.w0, 3, cfl=0.8, dt_every=10)
    assert np.all(field_err(w, ref) < STEP_TOL)


def test_conservation_and_stats_on_gpu(s2):
    """Inviscid periodic hybrid run: the volume integrals of all five
    conserved variables stay constant to round-off; stats match numpy."""
    nx, ny, nz = 40, 36, 32
    w0 = W.smooth_periodic(nx, ny, nz, seed=9, mach=0.8, amp_u=0.7, amp_s=0.2)
    L = 2 * np.pi
    with s2.Solver(nx, ny, nz, L, L, L, mach=0.8, re=-1.0, weno_order=5, threshold=0.1, cfl=0.5,
                   dt_every=1) as sv:
        sv.set_state(w0)
        s0 = sv.stats()
        dv = (L / nx) * (L / ny) * (L / nz)
        assert abs(s0["mass"] - w0[0].sum() * dv) < 1e-12 * abs(s0["mass"])
        assert abs(s0["energy"] - w0[4].sum() * dv) < 1e-12 * abs(s0["energy"])
        sv.step(20)
        s1 = sv.stats()
        assert s1["weno_frac"] > 0
    for key in ("mass", "energy"):
        assert abs(s1[key] - s0[key]) < 1e-12 * abs(s0[key])
    for a in range(3):
        assert abs(s1["mom"][a] - s0["mom"][a]) < 1e-12 * (abs(s0["mass"]) + abs(s0["mom"][a]))


def test_checkpoint_restart_bit_exact(s2):
    c = channel_small(48, 32, 24, seed=3)
    kw = case_kw(c)
    with s2.Solver.from_case(c, cfl=0.8, dt_every=4) as a:
        a.set_state(c.w0)
        a.step(10)
        wa = a.get_state()
        sa = a.stats()
    with s2.Solver.from_case(c, cfl=0.8, dt_every=4) as b:
        b.set_state(c.w0)
        b.step(5)
        mid = b.get_state()
        sb = b.stats()
    with s2.Solver.from_case(c, cfl=0.8, dt_every=4) as r:
        r.set_state(mid)
        r.set_clock(sb["t"], sb["step"], sb["dt"])
        r.step(5)
        wr = r.get_state()
        sr = r.stats()
    assert np.array_equal(wa, wr)
    assert sa["t"] == sr["t"] and sa["step"] == sr["step"]
    del kw


def test_device_pointers_and_stream(s2):
    """State in/out through torch CUDA tensors on a caller stream."""
    c = W.taylor_green(24)
    st = torch.cuda.Stream()
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3, stream=st.cuda_stream) as sv:
        wd = torch.from_numpy(c.w0).cuda()
        sv.set_state(wd)
        sv.step(2)
        out = torch.empty_like(wd)
        sv.get_state(out)
        wh = sv.get_state()
    assert np.array_equal(out.cpu().numpy(), wh)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stream_states_equal_set_step_get(s2, precision):
    """s2_stream_states, whose copies overlap the steps, gives state by state
    exactly what s2_set_state / s2_step / s2_get_state give in sequence: a
    pinned host stack, then one reused input, then device tensors."""
    c = channel_small(48, 32, 24, seed=5)
    ins = np.stack([channel_small(48, 32, 24, seed=5 + j).w0 for j in range(3)])
    nsteps = 4
    kw = dict(cfl=0.8, dt_every=3, precision=precision)
    with s2.Solver.from_case(c, **kw) as a:
        ref = []
        for j in range(3):
            a.set_state(ins[j])
            a.step(nsteps)
            ref.append(a.get_state())
        for _ in range(2):
            a.set_state(ins[0])
            a.step(nsteps)
        ref_last = a.get_state()
        st_a = a.stats()
    with s2.Solver.from_case(c, **kw) as b:
        pin_in = torch.from_numpy(ins).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        b.stream_states(pin_in, pin_out, nsteps)
        last = np.empty_like(ins[0])
        b.stream_states(ins[0], last, nsteps, count=2)  # staging buffers reused, stride 0 in and out
        st_b = b.stats()
        with pytest.raises(s2.S2Error) as ei:
            s2.s2_stream_states(b.h, ins, 0, last, 0, -1, nsteps)
        assert ei.value.code == s2.S2_EINVAL
    for j in range(3):
        assert np.array_equal(pin_out[j].numpy(), ref[j]), j
    assert np.array_equal(last, ref_last)
    assert st_a["step"] == st_b["step"] == 5 * nsteps and st_a["t"] == st_b["t"]
    with s2.Solver.from_case(c, **kw) as d:
        tin = torch.from_numpy(ins).cuda()
        tout = torch.empty_like(tin)
        d.stream_states(tin, tout, nsteps)
    assert np.array_equal(tout.cpu().numpy(), pin_out.numpy())


def test_stream_states_reports_an_invalid_state(s2):
    """A non-positive density in one streamed state makes the call return
    S2_ENONFINITE; every result is still copied out (the one before it equal
    to a sequential step), and the next call starts with a clear status."""
    c = W.taylor_green(16)
    bad = c.w0.copy()
    bad[0, 3, 4, 5] = -1.0
    ins = np.stack([c.w0, bad, c.w0])
    outs = np.full_like(ins, np.nan)
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3) as a:
        a.set_state(c.w0)
        a.step(1)
        ref = a.get_state()
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3) as sv:
        with pytest.raises(s2.S2Error) as ei:
            sv.stream_states(ins, outs, 1)
        assert ei.value.code == s2.S2_ENONFINITE
        assert np.array_equal(outs[0], ref)
        assert not np.isnan(outs[2]).all()
        again = np.empty_like(ins[:1])
        sv.stream_states(ins[:1], again, 1)


def test_nonfinite_state_reported(s2):
    c = W.taylor_green(16)
    w = c.w0.copy()
    w[0, 3, 4, 5] = -1.0  # negative density
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3) as sv:
        sv.set_state(w)
        sv.step(1)  # asynchronous: the error surfaces at the next sync
        with pytest.raises(s2.S2Error) as ei:
            sv.sync()
        assert ei.value.code == s2.S2_ENONFINITE
        # a valid state clears the status
        sv.set_state(c.w0)
        sv.step(1)
        sv.sync()


@pytest.mark.parametrize("orders", [(2, 2, 1), (4, 4, 3), (8, 8, 7), (8, 2, 5), (2, 8, 3), (6, 4, 0)])
def test_scheme_variants_rhs_parity(s2, orders):
    """Central orders 2/4/6/8, viscous orders 2/4/6/8 and WENO 1/3/5/7
    (the paper's C2-C8, V2-V8, W1-W7 sweep) on a ragged, stretched,
    periodic grid: RHS and flags match the oracle."""
    co, vo, wo = orders
    nx, ny, nz = 37, 29, 19
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=60 + co + vo, mach=0.7, amp_u=0.7, amp_s=0.25)
    xi = np.arange(ny) * L / ny
    kw = dict(y=xi + 0.25 * np.sin(xi), mach=0.7, re=150.0, weno_order=wo, threshold=0.15,
              central_order=co, visc_order=vo)
    e, f, of = rhs_parity(s2, w0, nx, ny, nz, L, L, L, **kw)
    assert np.all(e < RHS_TOL), e
    if wo:
        for a, b in zip(f, of):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("orders", [(4, 4, 3), (8, 8, 7)])
def test_scheme_variants_channel_10_steps(s2, orders):
    """Walls, stretched y, forcing, hybrid WENO at other orders: states
    after 10 steps match the oracle."""
    co, vo, wo = orders
    c = W.channel(48, 40, 24, seed=13)
    kw = case_kw(c)
    kw.update(central_order=co, visc_order=vo, weno_order=wo, threshold=0.05)
    sv, pr = make(s2, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cfl=0.8, dt_every=10, **kw)
    with sv:
        sv.set_state(c.w0)
        sv.step(10)
        w = sv.get_state()
    ref, _, _ = O.step(pr, c.w0, 10, cfl=0.8, dt_every=10)
    err = field_err(w, ref)
    print("orders %s: state error after 10 steps" % (orders,), err)
    assert np.all(err < STEP_TOL), err


@pytest.mark.parametrize("keep,orders", [(-1, (6, 6, 0)), (-1, (8, 6, 5)), (3, (6, 6, 7)), (1, (4, 4, 0)),
                                         (-1, (2, 2, 3))])
def test_keep_rhs_parity(s2, keep, orders):
    """KEEP-n central flux (exact logarithmic means, and n = 1, 3 series
    terms), central only and hybrid with WENO, on a ragged stretched
    periodic grid: RHS and flags match the oracle."""
    co, vo, wo = orders
    nx, ny, nz = 37, 29, 19
    L = 2 * np.pi
    w0 = W.smooth_periodic(nx, ny, nz, seed=70 + co + wo, mach=0.7, amp_u=0.7, amp_s=0.25)
    xi = np.arange(ny) * L / ny
    kw = dict(y=xi + 0.25 * np.sin(xi), mach=0.7, re=150.0, weno_order=wo, threshold=0.15,
              central_order=co, visc_order=vo, keep=keep)
    e, f, of = rhs_parity(s2, w0, nx, ny, nz, L, L, L, **kw)
    assert np.all(e < RHS_TOL), e
    if wo:
        for a, b in zip(f, of):
            assert np.array_equal(a, b)


def test_keep_channel_10_steps_and_entropy(s2):
    """KEEP with walls, stretched y, forcing and hybrid WENO5: states after
    10 steps match the oracle.  Inviscid, central and periodic, the GPU's
    RHS conserves the entropy -rho s/(gamma-1) to rounding (sum of v . R dV,
    v the entropy variables), as the oracle's does."""
    c = W.channel(48, 40, 24, seed=13)
    kw = case_kw(c)
    kw.update(weno_order=5, threshold=0.05, keep=-1)
    sv, pr = make(s2, c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cfl=0.8, dt_every=10, **kw)
    with sv:
        sv.set_state(c.w0)
        sv.step(10)
        w = sv.get_state()
    ref, _, _ = O.step(pr, c.w0, 10, cfl=0.8, dt_every=10)
    err = field_err(w, ref)
    print("KEEP channel: state error after 10 steps", err)
    assert np.all(err < STEP_TOL), err
    # entropy of the inviscid central GPU RHS
    nx, ny, nz = 30, 26, 22
    L = 2 * np.pi
    xi = np.arange(ny) * L / ny
    y = xi + 0.25 * np.sin(xi)
    w0 = W.smooth_periodic(nx, ny, nz, seed=41, mach=0.5, amp_u=0.6, amp_s=0.3)
    sv, pr = make(s2, nx, ny, nz, L, L, L, cfl=0.0, dt_fixed=1e-3, y=y, mach=0.5, re=-1.0, weno_order=0, keep=-1)
    with sv:
        sv.set_state(w0)
        r = sv.rhs()
    rho = w0[0]
    u, v, ww = w0[1] / rho, w0[2] / rho, w0[3] / rho
    q2 = u * u + v * v + ww * ww
    p = 0.4 * (w0[4] - 0.5 * rho * q2)
    s = np.log(p) - 1.4 * np.log(rho)
    b = rho / p
    ev = np.stack([(1.4 - s) / 0.4 - 0.5 * b * q2, b * u, b * v, b * ww, -b])
    ey, _ = O.metric(pr)
    prod = np.sum(ev * r, axis=0) * (1.0 / ey)[None, :, None]
    rel = abs(np.sum(prod)) / np.sum(np.abs(prod))
    print("KEEP entropy production of the GPU RHS (relative):", rel)
    assert rel < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stalled_copy_reported_as_timeout(s2, monkeypatch, precision):
    """Failure detection without a fault: with S2_TEST_STALL_COPIES=1 every
    staging barrier of the convective kernels expects 16 bytes more than
    its tensor-memory copies deliver (a completion that never comes), the
    kernels' bounded waits (20 ms) run out, the kernels return, and the
    step reports S2_ETIMEOUT.  The context stays usable: a solver created
    afterwards steps normally and matches a clean run."""
    c = W.taylor_green(16)
    monkeypatch.setenv("S2_TEST_STALL_COPIES", "1")
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3, precision=precision) as sv:
        sv.set_state(c.w0)
        sv.step(1)
        with pytest.raises(s2.S2Error) as ei:
            sv.sync()
        assert ei.value.code == s2.S2_ETIMEOUT
    monkeypatch.delenv("S2_TEST_STALL_COPIES")
    with s2.Solver.from_case(c, cfl=0.0, dt_fixed=1e-3, precision=precision) as sv:
        sv.set_state(c.w0)
        sv.step(2)
        sv.sync()
        w = sv.get_state()
    assert np.all(np.isfinite(w))
