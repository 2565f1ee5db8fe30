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


def test_tile_variants_give_identical_results(s2):
    c = W.channel(40, 36, 24, seed=2)
    out = []
    for tiles in ([0, 0, 0], [1, 1, 1], [1, 0, 1]):
        with s2.Solver.from_case(c, cfl=0.8, threshold=0.05) as sv:
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
