"""The bounds-checked build (libs2_checked.so, -DS2_CHECKED): every
kernel tests its index arithmetic against the array before each access
and reports S2_EBOUNDS instead of touching memory out of range
(compute-sanitizer is not available, so this stands in for it).  The
parity tests on small grids whose sizes are multiples of no tile -- odd
sizes, 1-point dimensions, walls, every stencil order, WENO 5 and 7, FP64
and mixed, the thermally perfect gas -- run again against the checked
library in a child process: they must pass with no bounds report."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SELECTION = ("ragged or scheme_variants_rhs or channel_small or weno7 or double_sod or "
             "mixed_rhs_ragged or mixed_rhs_orders or nonfinite or stalled")


def test_parity_cases_under_the_bounds_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05494_gb300 import build
    build.build()
    assert os.path.exists(build.LIB_CHECKED)
    env = dict(os.environ, S2_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "gpu",
                        "tests/test_gpu_parity.py", "tests/test_gpu_mixed.py", "tests/test_gpu_thermo.py",
                        "-k", SELECTION + " or thermally_perfect or primitive_fields"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
