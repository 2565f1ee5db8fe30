"""Host-side logic that needs no GPU: serving workload generation, arrival
process, autotuner choice and cache, and the error bound behind the
single-precision pre-test of the double-precision sensor decision, and the
roofline arithmetic of the bench line."""
import numpy as np
import pytest

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


def test_fast_division_exact(tmp_path):
    """The multiply-high division the kernels split point and slot indices
    with (FastDiv in the kernels' shared header, host build of the same
    code) equals integer division: every divisor up to 1100 and the grid
    extents' neighbourhood of powers of two, dividends at 0, near every
    multiple boundary sampled, random, and at 2^32 - 1."""
    import os
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "fastdiv.cu"
    src.write_text(r'''
#include <cstdio>
#include <cstdlib>
#include "s2_internal.cuh"
int main() {
  unsigned divs[2000];
  int nd = 0;
  for (unsigned d = 1; d <= 1100; ++d) divs[nd++] = d;
  for (int e = 11; e <= 31; ++e)
    for (int o = -2; o <= 2; ++o) divs[nd++] = (1u << e) + o;
  unsigned long long seed = 12345;
  long long checked = 0;
  for (int a = 0; a < nd; ++a) {
    s2::FastDiv f;
    f.init(divs[a]);
    const unsigned d = divs[a];
    unsigned ns[64];
    int k = 0;
    ns[k++] = 0; ns[k++] = 1; ns[k++] = 0xffffffffu; ns[k++] = 0xfffffffeu; ns[k++] = 0x7fffffffu;
    for (int r = 0; r < 30; ++r) {
      seed = seed * 6364136223846793005ull + 1442695040888963407ull;
      unsigned x = (unsigned)(seed >> 32);
      ns[k++] = x;
      unsigned q = x / d;
      if (q > 0) ns[k++] = q * d - 1;
      if (q > 0) ns[k++] = q * d;
    }
    for (int b = 0; b < k; ++b) {
      ++checked;
      if (f.div(ns[b]) != ns[b] / d) { printf("FAIL d=%u n=%u got %u\n", d, ns[b], f.div(ns[b])); return 1; }
    }
  }
  printf("ok %lld\n", checked);
  return 0;
}
''')
    exe = tmp_path / "fastdiv"
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", root + "/paper_2304_05494_gb300/csrc", "-I", root + "/include",
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr


def _sensor_pretest(g, th, thr2):
    """Single-precision pre-test of the double-precision sensor decision,
    step by step as the gradient kernel forms it (float32 arithmetic,
    round to nearest, no fused operations): returns (decided, on)."""
    f = np.float32
    a1, b1 = f(g[2][1]), f(g[1][2])
    a2, b2 = f(g[0][2]), f(g[2][0])
    a3, b3 = f(g[1][0]), f(g[0][1])
    thf, t2 = f(th), f(thr2)
    o1, o2, o3 = a1 - b1, a2 - b2, a3 - b3
    om2 = o1 * o1 + o2 * o2 + o3 * o3
    th2 = thf * thf
    m = th2 - t2 * (th2 + om2 + f(1))
    s1, s2, s3 = abs(a1) + abs(b1), abs(a2) + abs(b2), abs(a3) + abs(b3)
    scale = th2 + t2 * (th2 + (s1 * s1 + s2 * s2 + s3 * s3) + f(1))
    if abs(m) > f(2.0 ** -19) * scale:
        return True, bool(thf < 0 and m > 0)
    return False, None


def test_sensor_single_precision_pretest_matches_exact_decision():
    """Wherever the single-precision pre-test of the sensor decides, its
    decision is the exact one (margin th^2 - thr^2 (th^2 + |omega|^2 + 1)
    in rational arithmetic), on random gradients of many magnitudes, with
    strong cancellation in the vorticity, and on states placed within
    1e-3 .. 1e-9 of the threshold; close states fall back to double."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(7)
    decided = fallback = 0
    for it in range(6000):
        thr = [0.05, 0.2, 0.5, 0.0][it % 4]
        scale = 10.0 ** rng.uniform(-4, 4)
        g = rng.normal(size=(3, 3)) * scale
        if it % 3 == 1:  # cancellation: o_k small against its two gradients
            for a, b in ((2, 1), (0, 2), (1, 0)):
                g[b][a] = g[a][b] * (1 + rng.normal() * 1e-6)
        om2 = (g[2][1] - g[1][2]) ** 2 + (g[0][2] - g[2][0]) ** 2 + (g[1][0] - g[0][1]) ** 2
        if it % 2 == 0 and thr > 0:  # theta near the threshold
            th = -np.sqrt(thr * thr * (om2 + 1.0) / (1.0 - thr * thr)) * (1 + rng.choice([-1, 1]) * 10.0 ** rng.uniform(-9, -3))
        else:
            th = rng.normal() * scale
        thr2 = thr * thr
        o = [Fr(g[2][1]) - Fr(g[1][2]), Fr(g[0][2]) - Fr(g[2][0]), Fr(g[1][0]) - Fr(g[0][1])]
        T = Fr(th)
        exact_m = T * T - Fr(thr2) * (T * T + sum(x * x for x in o) + 1)
        exact_on = th < 0 and exact_m > 0
        ok, on = _sensor_pretest(g, th, thr2)
        if ok:
            decided += 1
            assert on == exact_on, (g, th, thr)
        else:
            fallback += 1
    assert decided > 4000 and fallback > 0


def test_bench_roofline_arithmetic(monkeypatch):
    """The bench line's roofline objects from a synthetic per-class profile
    (total ms and launches per kernel class): achieved = algorithmic bytes
    (flops) per launch over the mean launch time, the dominant class is the
    one with the most time, the step fraction uses the method's 480 B per
    point-step, and the whole-job rate sums the replicas' work."""
    import bench
    monkeypatch.setattr(bench, "hbm_peak_gbs", lambda: (6000.0, "measured"))

    class Case:
        points = 1_000_000
        nx = ny = nz = 100

    prof = {"prims": (6.0, 6), "visc": (30.0, 6), "update": (12.0, 6), "flux_x": (9.0, 6), "grad": (3.0, 6)}
    r = bench.mixed_roofline(Case, prof, step_ms=20.0)
    assert r["kernel"] == "visc" and r["bound"] == "hbm"
    assert r["per_launch_ms"] == 5.0
    assert r["achieved"] == pytest.approx(bench.MIXED_BYTES["visc"] * 1e6 / 5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["step_frac"] == pytest.approx(480.0 * 1e6 / 20e-3 / 1e9 / 6000.0)
    assert r["frac_per_kernel"]["update"] == round(bench.MIXED_BYTES["update"] * 1e6 / 2e-3 / 1e9 / 6000.0, 3)
    assert r["traffic"] == pytest.approx(bench.MIXED_DRAM_BYTES["visc"] * 1e6)

    f = bench.fp64_roofline(Case, {"visc": (60.0, 6), "prims": (10.0, 6)}, 2, 0.0, 50.0, 1250.0)
    assert f["kernel"] == "visc" and f["bound"] == "alu"
    assert f["achieved"] == pytest.approx(bench.ALG_FLOPS["visc"] * 1e6 / 10e-3 / 1e9)
    assert f["frac"] == pytest.approx(f["achieved"] / bench.FP64_PEAK_GFLOPS)
    assert f["frac_of_fma_measured"] == pytest.approx(f["achieved"] / 1250.0)
    assert bench.whole_job_rate(1e6, 10, 2, 100.0) == pytest.approx(2e8)
