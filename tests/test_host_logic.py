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
