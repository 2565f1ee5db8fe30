"""Host-side logic that needs no GPU: serving workload generation, arrival
process, autotuner choice and cache."""
import numpy as np

from paper_2304_05494_gb300 import autotune, serve


def test_request_generator_ranges_and_seed():
    a = serve.make_requests(200, seed=3)
    b = serve.make_requests(200, seed=3)
    assert [(r.n, r.steps, r.mach) for r in a] == [(r.n, r.steps, r.mach) for r in b]
    assert {r.n for r in a} <= set(serve.SIZES) and len({r.n for r in a}) == len(serve.SIZES)
    assert all(100 <= r.steps <= 1000 for r in a)
    assert all(0.1 <= r.mach <= 0.8 and 400 <= r.re <= 3200 for r in a)
    assert {r.kind for r in a} == {"tgv", "turb"}


def test_poisson_arrivals_rate():
    reqs = serve.make_requests(4000, seed=1)
    serve.poisson_arrivals(reqs, rate=50.0, seed=2)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0


def test_autotune_choice_and_cache(tmp_path):
    times = {0: {"flux_x": 1.0, "flux_y": 2.0, "flux_z": 3.0}, 1: {"flux_x": 2.0, "flux_y": 1.0, "flux_z": 3.5}}
    assert autotune.choose(times) == [0, 1, 0]
    p = str(tmp_path / "c.json")
    autotune.save_cache({"k": {"tiles": [0, 1, 0]}}, p)
    assert autotune.load_cache(p)["k"]["tiles"] == [0, 1, 0]
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    assert autotune.key((32, 48, 64), "mixed", 5, "G").startswith("32x48x64|mixed|weno5|G")
