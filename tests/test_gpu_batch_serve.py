"""Batched stepping, tile autotuning and the serving loop on the GPU.

A box's results must not depend on what else runs with it: members of a
batch (one graph launch per step, members as concurrent branches) and
requests served in a continuous-batching mix must match their solo runs
bit for bit (the kernels are deterministic and share no buffers), and
the CPU oracle run on the same box: FP64 members to 1e-11 per conserved
field, mixed-precision members to 3e-4 of the FP64 oracle.  The tile shape
of the flux kernels must not change results either.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W

TOL_FP64 = 1e-11   # field-normalised, FP64 members against the oracle
TOL_MIXED = 3e-4   # field-normalised, mixed members against the FP64 oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import s2 as mod
    return mod


def solo(s2, case, steps, **kw):
    with s2.Solver.from_case(case, **kw) as sv:
        sv.set_state(case.w0)
        sv.step(steps)
        return sv.get_state()


def oracle_steps(case, steps, cfl=None, dt_every=None, threshold=None):
    """The CPU oracle's state after the given steps from case.w0, with the
    solver's dt schedule (CFL every dt_every steps)."""
    pr = O.Problem(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, y=case.y, gamma=case.gamma,
                   prandtl=case.prandtl, mach=case.mach, re=case.re, visc_exp=case.visc_exp, t_ref=case.t_ref,
                   wall_y=case.wall_y, t_wall=case.t_wall, force=case.force, weno_order=case.weno_order,
                   threshold=case.threshold if threshold is None else threshold)
    w, _, _ = O.step(pr, case.w0, steps, cfl=case.cfl if cfl is None else cfl,
                     dt_every=case.dt_every if dt_every is None else dt_every)
    return w


def field_err(a, b):
    return float(np.max(np.max(np.abs(a - b), axis=(1, 2, 3)) / np.max(np.abs(b), axis=(1, 2, 3))))


def test_batch_members_match_solo_runs(s2):
    cases = [(W.taylor_green(24), dict(precision="fp64", cfl=0.8, dt_every=3)),
             (W.channel(48, 32, 16, seed=8), dict(precision="mixed", cfl=0.8, dt_every=2)),
             (W.isotropic(32, mach_t=0.7, seed=5, weno_order=5), dict(precision="fp64", cfl=0.6, dt_every=4,
                                                                     threshold=0.05))]
    solvers = []
    for c, kw in cases:
        sv = s2.Solver.from_case(c, **kw)
        sv.set_state(c.w0)
        solvers.append(sv)
    with s2.Batch(solvers) as b:
        b.step(4)
        b.step(2)
        b.sync()
    got = [sv.get_state() for sv in solvers]
    stats = [sv.stats() for sv in solvers]
    for sv in solvers:
        sv.close()
    for (c, kw), g, st in zip(cases, got, stats):
        assert st["step"] == 6
        assert np.array_equal(g, solo(s2, c, 6, **kw))
        ref = oracle_steps(c, 6, cfl=kw["cfl"], dt_every=kw["dt_every"], threshold=kw.get("threshold"))
        tol = TOL_FP64 if kw["precision"] == "fp64" else TOL_MIXED
        assert field_err(g, ref) < tol, (c.name, kw["precision"], field_err(g, ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_worklist_batch_of_uneven_boxes_matches_solo_runs(s2, precision):
    """Work-list batching: boxes of different sizes and shapes sharing their
    kernels run as one group (each kernel one launch for all of them, the
    work list giving every CTA its box and tile); every member equals its
    solo run bit for bit, and the whole step costs the launches of one box.
    A member with another scheme (too few for a group of its own) keeps its
    own launch sequence."""
    box = W.Case(name="smooth28x20x12", nx=28, ny=20, nz=12, lx=2 * np.pi, ly=2 * np.pi, lz=2 * np.pi,
                 w0=W.smooth_periodic(28, 20, 12, seed=7, mach=0.5, amp_u=0.4, amp_s=0.1), mach=0.5, re=300.0)
    cases = [W.taylor_green(24, seed=3), W.taylor_green(32, mach=0.4, re=800.0, seed=4),
             W.isotropic(20, mach_t=0.6, seed=6, weno_order=5), box]
    for c in cases:
        c.weno_order, c.threshold, c.cfl, c.dt_every = 5, 0.1, 0.8, 2
    odd = W.channel(40, 24, 16, seed=9)  # walls and forcing: another kernel set
    kw = dict(precision=precision)
    solvers = []
    for c in cases + [odd]:
        sv = s2.Solver.from_case(c, **kw)
        sv.set_state(c.w0)
        solvers.append(sv)
    with s2.Batch(solvers) as b:
        n_work = b.launches_per_step
        b.step(3)
        b.sync()
    got = [sv.get_state() for sv in solvers]
    for sv in solvers:
        sv.close()
    for c, g in zip(cases + [odd], got):
        assert np.array_equal(g, solo(s2, c, 3, **kw)), c.name
    # the branch graph launches every member's kernels; the work list one
    # set for the group and the odd member's own
    solvers = [s2.Solver.from_case(c, **kw) for c in cases + [odd]]
    with s2.Batch(solvers, mode="branches") as b:
        n_branch = b.launches_per_step
    for sv in solvers:
        sv.close()
    assert n_work < n_branch / 2, (n_work, n_branch)
    assert n_work <= 2 * 45


@pytest.mark.parametrize("precision,sizes,factor", [
    ("mixed", [16] * 16 + [24] * 32 + [32] * 8, 0.8),
    ("fp64", [16] * 48 + [24] * 16, 0.9)])
def test_worklist_batch_runs_many_small_boxes_faster(s2, precision, sizes, factor):
    """Many small boxes: the work list's one launch per kernel for all of
    them beats launching every member's kernels as graph branches."""
    import time
    cases = [W.taylor_green(n, mach=0.3, seed=10 + i) for i, n in enumerate(sizes)]
    for c in cases:
        c.weno_order, c.threshold = 5, 0.2
    times = {}
    for mode in ("branches", "worklist", "branches", "worklist"):
        solvers = []
        for c in cases:
            sv = s2.Solver.from_case(c, precision=precision)
            sv.set_state(c.w0)
            solvers.append(sv)
        with s2.Batch(solvers, mode=mode) as b:
            b.step(2)
            b.sync()
            t0 = time.perf_counter()
            b.step(10)
            b.sync()
            times[mode] = min(times.get(mode, 1e9), time.perf_counter() - t0)
        for sv in solvers:
            sv.close()
    assert times["worklist"] < factor * times["branches"], times


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tile_variants_give_identical_results(s2, precision):
    """Every flux tile shape (and, in single precision, its two-points-per-
    thread layout) gives bit-identical results on a grid that is a multiple
    of none of them."""
    c = W.channel(40, 36, 24, seed=2)
    out = []
    for tiles in ([0, 0, 0], [1, 1, 1], [1, 0, 1]):
        with s2.Solver.from_case(c, cfl=0.8, threshold=0.05, precision=precision) as sv:
            sv.set_tiles(tiles)
            sv.set_state(c.w0)
            sv.step(3)
            out.append(sv.get_state())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_autotuner_caches_a_choice(s2, tmp_path):
    from paper_2304_05494_gb300 import autotune
    c = W.taylor_green(32)
    c.weno_order, c.threshold = 5, 0.1
    path = str(tmp_path / "tiles.json")
    with s2.Solver.from_case(c, precision="mixed") as sv:
        t = autotune.tuning_for(sv, c.w0, (c.nx, c.ny, c.nz), "mixed", 5, path=path, steps=2)
        assert all(x in (0, 1) for x in t["tiles"])
        assert all(x in autotune.FLUX_CTAS for x in t["flux_ctas_per_sm"]) and t["z_planes"] in autotune.Z_PLANES
        assert t["weno_ctas_per_sm"] in autotune.WENO_CTAS
        assert sv.get_tuning() == t
        sv.step(1)  # the solver still runs after tuning
        sv.sync()
    cache = autotune.load_cache(path)
    assert len(cache) == 1 and list(cache.values())[0]["tuning"] == t
    # a second solver of the same class takes the cached choice without tuning
    with s2.Solver.from_case(c, precision="mixed") as sv:
        assert autotune.tiles_for(sv, c.w0, (c.nx, c.ny, c.nz), "mixed", 5, path=path) == t["tiles"]
        assert sv.get_tuning() == t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_knobs_give_identical_results(s2, precision):
    """CTAs per SM of the flux and WENO grids and z-planes per CTA of the
    z-marching passes change the launch shape, not the results.  The one
    exception: with channel forcing in single precision, the viscous
    z-pass sums the bulk forcing per CTA, so the plane count changes the
    order of that sum (results then agree to single-precision rounding)."""
    def run(c, **knobs):
        with s2.Solver.from_case(c, cfl=0.8, threshold=0.05, precision=precision) as sv:
            if knobs:
                sv.set_tuning(**knobs)
            sv.set_state(c.w0)
            sv.step(3)
            return sv.get_state()

    chan = W.channel(40, 36, 30, seed=2)
    ref = run(chan)
    for knobs in (dict(flux_ctas_per_sm=1, weno_ctas_per_sm=4), dict(flux_ctas_per_sm=[3, 0, 2], weno_ctas_per_sm=32)):
        assert np.array_equal(ref, run(chan, **knobs)), knobs
    zc = run(chan, z_planes=8)
    if precision == "fp64":
        assert np.array_equal(ref, zc)
    else:
        assert field_err(zc, ref) < 1e-6
    box = W.isotropic(24, mach_t=0.6, seed=3, weno_order=5)
    refb = run(box)
    for knobs in (dict(z_planes=4, flux_ctas_per_sm=2), dict(z_planes=24, weno_ctas_per_sm=8), dict(z_planes=16)):
        assert np.array_equal(refb, run(box, **knobs)), knobs


def test_serving_results_same_alone_and_in_the_mix(s2):
    from paper_2304_05494_gb300 import serve
    reqs = serve.make_requests(5, seed=11, sizes=(24, 32), steps=(12, 30), precisions=("mixed", "fp64"))
    for i, r in enumerate(reqs):
        r.arrival = 0.02 * i  # staggered: later requests join a running batch
    out = serve.Server(max_slots=3, steps_per_tick=4, keep_results=True).run(reqs)
    assert out["point_steps"] == sum(r.points * r.steps for r in reqs)
    assert np.isfinite(out["p50_step_latency_ms"]) and np.isfinite(out["p99_step_latency_ms"])
    assert out["throughput"] > 0
    for r in reqs:
        c = serve.initial_case(r)
        alone = solo(s2, c, r.steps, precision=r.precision)
        assert np.array_equal(r.result, alone), r.rid
        ref = oracle_steps(c, r.steps)
        tol = TOL_FP64 if r.precision == "fp64" else TOL_MIXED
        assert field_err(r.result, ref) < tol, (r.rid, r.precision, field_err(r.result, ref))


def test_serving_isolates_failed_and_cancelled_requests(s2):
    """Fault injection on the host side of the serving loop: one request
    starts from a state with a negative density (the device flags it:
    S2_ENONFINITE), one is cancelled by its client after 8 steps; both are
    retired while the batch keeps running, and the other requests' results
    are bit-identical to their solo runs."""
    from paper_2304_05494_gb300 import serve
    reqs = serve.make_requests(4, seed=21, sizes=(24, 32), steps=(16, 24), precisions=("fp64", "mixed"))
    for i, r in enumerate(reqs):
        r.arrival = 0.0
    reqs[1].corrupt = True
    reqs[2].cancel_after = 8
    out = serve.Server(max_slots=4, steps_per_tick=4, keep_results=True).run(reqs)
    assert reqs[1].status == "failed: " + s2.s2_strerror(s2.S2_ENONFINITE)
    assert reqs[2].status == "cancelled" and reqs[2].result is None
    assert out["failed"] == 1 and out["cancelled"] == 1 and out["done"] == 2
    for r in (reqs[0], reqs[3]):
        assert r.status == "done"
        alone = solo(s2, serve.initial_case(r), r.steps, precision=r.precision)
        assert np.array_equal(r.result, alone), r.rid


def test_allocation_failure_releases_everything(s2):
    """An allocator callback that runs dry part-way through s2_create: the
    call returns S2_ENOMEM and hands every block it did get back to the
    callback's free."""
    import ctypes as C
    torch = pytest.importorskip("torch")
    live = {}
    calls = {"alloc": 0}

    @s2._ALLOC
    def alloc(nbytes, ctx):
        calls["alloc"] += 1
        if calls["alloc"] > 6:
            return None
        p = torch.cuda.caching_allocator_alloc(max(int(nbytes), 16))
        live[p] = nbytes
        return p

    @s2._FREE
    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)
        del live[ptr]

    g = s2.s2_grid(24, 20, 16, 1.0, 1.0, 1.0)
    gas = s2.s2_gas(1.4, 0.72, 0.5, 100.0, 0.76, 1.0)
    b = s2.s2_bcs(0, 0, 0, 1.0, 0)
    sch = s2.s2_scheme(6, 5, 6, 0.2, 0, 0.8, 0.0, 10)
    dev = s2.s2_device()
    dev.alloc = alloc
    dev.free = free
    dev.device = -1
    h = C.c_void_p()
    rc = s2._lib.s2_create(C.byref(g), None, C.byref(gas), C.byref(b), C.byref(sch), C.byref(dev), C.byref(h))
    assert rc == s2.S2_ENOMEM
    assert calls["alloc"] > 6 and not live
