"""Throughput on the grid of the paper's single-GPU evaluation (Sec. 4.1,
420 x 250 x 320 = 33.6M points), for a direct comparison with the A100 and
MI250x iteration times its launch-bounds table prints for the central
scheme and for WENO everywhere (thread block 128 x 3).

The flow is the compressible channel of the benchmark (tanh-stretched y,
isothermal walls, bulk Mach 1.5) at that grid.  Scheme "central": central
6th order, sensor off; scheme "weno": WENO5 at every interface.  Each line
reports ms per RK3 step (one iteration = one full RK3 step, three RHS
stages) and grid-point RK3 steps per second, in FP64 and in mixed
precision.

  python -m paper_2304_05494_gb300.paper_grid [--steps 5]
"""
from __future__ import annotations

import argparse
import json
import time

from . import workloads as W

# The paper's figures (FP64): ms per iteration, launch-bounds table of
# Sec. 4.1 at a 128 x 3 thread block.
PAPER_MS = {("central", "A100"): 317.5, ("weno", "A100"): 476.4,
            ("central", "MI250x GCD"): 579.3, ("weno", "MI250x GCD"): 994.5}
NX, NY, NZ = 420, 250, 320


def time_steps(case, steps: int, **kw) -> float:
    from . import s2
    with s2.Solver.from_case(case, **kw) as sv:
        sv.set_state(case.w0)
        sv.step(2)
        sv.sync()
        t = time.perf_counter()
        sv.step(steps)
        sv.sync()
        return (time.perf_counter() - t) / steps * 1e3


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=5)
    args = ap.parse_args(argv)
    case = W.channel(NX, NY, NZ)
    n = NX * NY * NZ
    for scheme, kw in (("central", dict(weno_order=0)), ("weno", dict(weno_order=5, threshold=-1.0))):
        for precision in ("fp64", "mixed"):
            ms = time_steps(case, args.steps, precision=precision, **kw)
            print(json.dumps({"grid": [NX, NY, NZ], "scheme": scheme, "precision": precision,
                              "ms_per_step": ms, "point_steps_per_s": n / (ms * 1e-3),
                              "paper_fp64_ms_per_iteration": {hw: PAPER_MS[(scheme, hw)]
                                                              for hw in ("A100", "MI250x GCD")}}))


if __name__ == "__main__":
    main()
