"""The oracle's operation tally (oracle/tally.py), which gives the
algorithmic flop counts of the benchmark's double-precision roofline.

The counting build must compute exactly what the plain oracle computes, its
counts must match closed forms of the operations the oracle's direct
formulas perform, and the constants bench.py quotes must equal a fresh
tally.
"""
import numpy as np
import pytest

import bench
from oracle import oracle as O
from oracle import tally as TL
from paper_2304_05494_gb300 import workloads as W


def _channel_problem(case, **kw):
    return O.Problem(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, y=case.y, mach=case.mach, re=case.re,
                     visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y, t_wall=case.t_wall,
                     force=case.force, weno_order=case.weno_order, **kw)


@pytest.fixture(scope="module")
def case():
    return W.channel(32, 24, 16, seed=4)


def test_counting_build_is_bit_identical(case):
    """Same RHS, flags, dt and RK3 steps as the plain oracle."""
    pr = _channel_problem(case, threshold=0.05)
    r0, f0 = O.rhs(pr, case.w0, flags=True)
    w0, _, _ = O.step(pr, case.w0, 2, cfl=0.8)
    dt0 = O.dt(pr, case.w0, 0.8)
    (_, (r1, f1)) = TL.run(lambda: O.rhs(pr, case.w0, flags=True))
    (_, (w1, _, _)) = TL.run(lambda: O.step(pr, case.w0, 2, cfl=0.8))
    (_, dt1) = TL.run(lambda: O.dt(pr, case.w0, 0.8))
    assert np.array_equal(r0, r1) and all(np.array_equal(a, b) for a, b in zip(f0, f1))
    assert np.array_equal(w0, w1) and dt0 == dt1
    assert f0[0].any(), "the case should flag some interfaces"


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_central_interface_count_closed_form(order):
    """One split-form interface flux of order 2L as the oracle forms it:
    L(L+1)/2 pairs of 29 operations (six pair means, five triple products
    accumulated, the pressure sum), then per l five scaled accumulations
    (3 each) and the pressure term (2), and the pressure added to the normal
    momentum: 29 L(L+1)/2 + 17 L + 1."""
    L = order // 2
    n = 12
    w = W.smooth_periodic(n, n, n, seed=2, mach=0.5, amp_u=0.2, amp_s=0.05)
    pr = O.Problem(n, n, n, 1.0, 1.0, 1.0, mach=0.5, re=-1.0, central_order=order, visc_order=order)
    c, _ = TL.run(lambda: O.rhs(pr, w, terms=O.CONV))
    interfaces = 3 * (n + 1) * n * n
    # per direction and field: difference, scale, subtract; plus the
    # reciprocals 1/dx and 1/dz of the x and z scales
    per_point_diff = 3 * 5 * 3 + 2
    total = TL.flops(c["central"])
    assert total == interfaces * (29 * L * (L + 1) // 2 + 17 * L + 1) + n ** 3 * per_point_diff


def test_update_and_state_counts(case):
    """RK3 update: w += dt (gamma R + rho R_prev) is 5 operations per field;
    H and c cost 11 per point; the primitive recovery 14."""
    pr = _channel_problem(case, threshold=1e30)
    t = TL.per_point_step(pr, case.w0, 0.0)
    assert t["per_point_stage"]["update"] == 25.0
    assert t["h_and_c_per_point"] == 11.0
    assert t["per_point_stage"]["prims"] == 25.0


def test_bench_constants_equal_the_tally(case):
    """bench.py's algorithmic flop constants are the tally of the benchmark
    scheme (central 6, WENO5, viscous 6, calorically perfect gas)."""
    pr = _channel_problem(case, threshold=case.threshold)
    t = TL.per_point_step(pr, case.w0, 0.0)
    st = t["per_point_stage"]
    for k in ("prims", "grad", "visc", "update"):
        assert bench.ALG_FLOPS[k] == pytest.approx(st[k], rel=1e-12), k
    assert bench.ALG_FLOPS_CENTRAL_INTERFACE == t["central_interface"]
    assert bench.ALG_FLOPS_WENO_INTERFACE == t["weno_interface"]
    assert bench.ALG_FLOPS_FLUX_DIFFERENCE == pytest.approx(t["flux_difference_per_point"] / 3, rel=1e-12)
    assert bench.ALG_FLOPS_VISC_GRAD == pytest.approx(st["visc_grad"], rel=1e-12)
