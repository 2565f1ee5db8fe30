"""The allocation-free time-step entry point (s2_cfl_dt_noalloc).

It serves callers that cannot allocate device memory when they need a step
size (their memory belongs to a pooling allocator or another framework, or
their loop cannot afford cudaMalloc's synchronisation); its scratch is a
fixed array compiled into the library.  Here it is called through the C ABI
twice in a row, on two different problems, and each result is compared
with the dt that s2_step computes from the same state.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def s2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import s2 as mod
    return mod


def solver_dt(s2, case):
    """dt computed by s2_step at step 0 from the initial state."""
    with s2.Solver.from_case(case, cfl=0.8, dt_every=10) as sv:
        sv.set_state(case.w0)
        sv.step(1)
        return sv.stats()["dt"]


def noalloc_dt(s2, case, eta_y, w0=None):
    grid = s2.s2_grid(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz)
    gas = s2.s2_gas(case.gamma, case.prandtl, case.mach, case.re, case.visc_exp, case.t_ref)
    w = torch.from_numpy(case.w0 if w0 is None else w0).cuda()
    ey = torch.from_numpy(eta_y).cuda() if eta_y is not None else None
    dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    rc = s2.s2_cfl_dt_noalloc(grid, gas, w, ey, 0.8, dt, st.cuda_stream)
    assert rc == s2.S2_OK, s2.s2_strerror(rc)
    st.synchronize()
    return float(dt.item())


def test_noalloc_dt_matches_solver_twice_in_a_row(s2):
    tgv = W.taylor_green(24)
    chan = W.channel(48, 32, 16, seed=4)
    pr = O.Problem(chan.nx, chan.ny, chan.nz, chan.lx, chan.ly, chan.lz, y=chan.y, wall_y=True)
    eta_y, _ = O.metric(pr)
    ref_tgv = solver_dt(s2, tgv)
    ref_chan = solver_dt(s2, chan)
    a = noalloc_dt(s2, tgv, None)
    b = noalloc_dt(s2, chan, eta_y)
    assert abs(a - ref_tgv) <= TOL * ref_tgv, (a, ref_tgv)
    assert abs(b - ref_chan) <= TOL * ref_chan, (b, ref_chan)
    # the shared scratch keeps the previous call's partials; a repeat of
    # the first problem must not see them
    assert noalloc_dt(s2, tgv, None) == a


@pytest.mark.parametrize("bad", ["negative_density", "negative_energy", "nan_momentum"])
def test_noalloc_dt_is_zero_for_an_invalid_state(s2, bad):
    """A single point that s2_step would report as invalid makes dt = 0
    instead of a plausible value taken from the other points."""
    tgv = W.taylor_green(24)
    w = tgv.w0.copy()
    if bad == "negative_density":
        w[0, 3, 5, 7] = -w[0, 3, 5, 7]
    elif bad == "negative_energy":
        w[4, 3, 5, 7] = -1.0
    else:
        w[2, 3, 5, 7] = np.nan
    assert noalloc_dt(s2, tgv, None) > 0.0
    assert noalloc_dt(s2, tgv, None, w) == 0.0
    # and the next call on a valid state is unaffected by the shared scratch
    assert noalloc_dt(s2, tgv, None) > 0.0


def test_noalloc_rejects_grids_beyond_its_scratch(s2):
    grid = s2.s2_grid(2048, 1024, 1024, 1.0, 1.0, 1.0)
    gas = s2.s2_gas(1.4, 0.72, 0.5, 100.0, 0.76, 1.0)
    w = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: rejected first
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = s2.s2_cfl_dt_noalloc(grid, gas, w, None, 0.8, dt, None)
    assert rc == s2.S2_ETOOBIG
    assert "scratch" in s2.s2_strerror(rc)
    # extents whose product would overflow a 64-bit integer are rejected too
    big = 2 ** 31 - 1
    for ext in ((big, big, big), (1, big, big), (big, 1, 1)):
        rc = s2.s2_cfl_dt_noalloc(s2.s2_grid(*ext, 1.0, 1.0, 1.0), gas, w, None, 0.8, dt, None)
        assert rc == s2.S2_ETOOBIG, ext
