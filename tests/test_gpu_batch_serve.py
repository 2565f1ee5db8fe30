"""Batched stepping, tile autotuning and the serving loop on the GPU.

A box's results must not depend on what else runs with it: members of a
batch (one graph launch per step, members as concurrent branches) and
requests served in a continuous-batching mix must match their solo runs
bit for bit (the kernels are deterministic and share no buffers).  The
tile shape of the flux kernels must not change results either.
"""
import numpy as np
import pytest

from paper_2304_05494_gb300 import workloads as W

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
    path = str(tmp_path / "tiles.json")
    with s2.Solver.from_case(c, precision="mixed") as sv:
        tiles = autotune.tiles_for(sv, c.w0, (c.nx, c.ny, c.nz), "mixed", 0, path=path, steps=2)
        assert all(t in (0, 1) for t in tiles)
        sv.step(1)  # the solver still runs after tuning
        sv.sync()
    cache = autotune.load_cache(path)
    assert len(cache) == 1 and list(cache.values())[0]["tiles"] == tiles


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
