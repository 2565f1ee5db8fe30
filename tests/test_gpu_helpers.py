"""The solver's hand-written numeric helpers against CUDA's own results
over sweeps that include the switch points and special values:

* rcp_pos: 1/x from a single-precision seed and two Newton-Raphson steps,
  claimed within 1 ulp of 1/x, the library division outside [2^-100, 2^100];
* d2f_int / f2d_int: double <-> float on the integer pipe, claimed to round
  to nearest with ties away from zero (the hardware rounds ties to even),
  to flush results below the normal range to signed zero, to saturate to
  infinity, and to convert float -> double exactly;
* the power law mu = x^(p/q) by one Halley step from a single-precision
  seed, claimed to reach double precision.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("helpers") / "libs2_helpers.so")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(os.path.dirname(HERE), "include"),
                    os.path.join(HERE, "gpu_helpers.cu"), "-o", out], check=True)
    lb = C.CDLL(out)
    lb.helpers_run.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int]
    lb.helpers_run.restype = C.c_int
    return lb


def run(lib, which, x, p=19, q=25):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    dp = C.POINTER(C.c_double)
    assert lib.helpers_run(which, x.ctypes.data_as(dp), out.ctypes.data_as(dp), x.size, p, q) == 0
    return out


def ulps(a, b):
    """|a - b| in units of the last place of b (double)."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_rcp_pos_within_one_ulp(lib):
    rng = np.random.default_rng(1)
    e = np.concatenate([np.linspace(-300, 300, 20001), [-101, -100, -99.9999, 99.9999, 100, 100.5, 101]])
    x = np.concatenate([2.0 ** e, 2.0 ** e * rng.uniform(1, 2, e.size), [2.0 ** -1022, 1e-300, 1e300, 1.0, 3.0]])
    r = run(lib, 0, x)
    assert np.all(ulps(r, 1.0 / x) <= 1.0), np.max(ulps(r, 1.0 / x))
    # inside the seed's range the result is usually the correctly rounded one
    inside = (x > 2.0 ** -99) & (x < 2.0 ** 99)
    assert np.mean(r[inside] == 1.0 / x[inside]) > 0.99


def test_d2f_int_rounding_flush_and_saturation(lib):
    rng = np.random.default_rng(2)
    f32 = np.finfo(np.float32)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-37, 38, 20000),
                        [0.0, -0.0, 1.0, -1.0, float(f32.max), -float(f32.max), float(f32.tiny),
                         1e39, -1e39, np.inf, -np.inf, 1e-40, -1e-40, 2.0 ** -150]])
    mine = run(lib, 1, x)
    hw = run(lib, 2, x)
    normal = (np.abs(hw) >= float(f32.tiny)) & np.isfinite(hw)
    diff = normal & (mine != hw)
    # only exact ties (the dropped 29 bits are 1000...0) may differ, and there
    # the integer path rounds away from zero
    bits = x.view(np.uint64)
    tie = (bits & np.uint64((1 << 29) - 1)) == np.uint64(1 << 28)
    assert np.all(tie[diff])
    assert np.all(np.abs(mine[diff]) > np.abs(x[diff]))
    # ties constructed on purpose: halfway between two floats
    f = rng.uniform(1, 2, 1000).astype(np.float32).astype(np.float64)
    half = f + np.spacing(f.astype(np.float32)).astype(np.float64) / 2
    assert np.all(run(lib, 1, half) == (f + np.spacing(f.astype(np.float32)).astype(np.float64)))
    # results below the normal range flush to signed zero, above saturate
    small = (np.abs(x) < float(f32.tiny) / 2) & (x != 0)
    assert np.all(mine[small] == 0) and np.all(np.signbit(mine[small]) == np.signbit(x[small]))
    big = np.abs(x) > 3.5e38
    assert np.all(np.isinf(mine[big])) and np.all(np.sign(mine[big]) == np.sign(x[big]))


def test_f2d_int_exact_for_floats(lib):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-37, 38, 20000), [0.0, -0.0, 1e-40]])
    back = run(lib, 3, x)  # float(x) by the hardware, then back to double on the integer pipe
    ref = x.astype(np.float32).astype(np.float64)
    normal = np.abs(ref) >= float(np.finfo(np.float32).tiny)
    assert np.array_equal(back[normal], ref[normal])
    assert np.all(back[~normal] == 0)


@pytest.mark.parametrize("p,q", [(19, 25), (3, 4), (2, 3)])
def test_halley_power_law_reaches_double_precision(lib, p, q):
    x = np.concatenate([np.geomspace(0.05, 20.0, 20001), [1.0, 0.5, 2.0]])
    mine = run(lib, 4, x, p, q)
    ref = run(lib, 5, x, p, q)  # CUDA's pow in double precision
    rel = np.abs(mine - ref) / ref
    assert np.max(rel) < 9e-16, np.max(rel)  # 4 ulp: the step's own rounding and pow's (measured <= 2.7)
