"""Error statement of the mixed path against the FP64 path on one workload.

Runs the same initial state for N RK3 steps in FP64 and in mixed precision
(single-precision flux/WENO/viscous arithmetic, double-precision state and
E -> T recovery) and prints one JSON line with the per-field error of the
mixed state against the FP64 state (max |a-b| / max |b| per conserved
field), the total energy of both runs and its drift, and the time per step
of each.

  python -m paper_2304_05494_gb300.precision_report --config channel1024 --steps 100
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W

CONFIGS = {
    "tgv32": lambda: W.taylor_green(32),
    "channel256": lambda: W.channel(),
    "isotropic512": lambda: W.isotropic(512),
    "channel1024": lambda: W.channel_big(),
}


def run(case, precision: str, steps: int):
    from . import s2
    import torch
    with s2.Solver.from_case(case, precision=precision) as sv:
        sv.set_state(case.w0)
        e0 = sv.stats()["energy"]
        sv.step(1)
        sv.sync()
        t = time.perf_counter()
        sv.step(steps - 1)
        sv.sync()
        ms = (time.perf_counter() - t) / max(steps - 1, 1) * 1e3
        st = sv.stats()
        w = sv.get_state()
    torch.cuda.empty_cache()
    return w, st, e0, ms


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="channel256", choices=sorted(CONFIGS))
    ap.add_argument("--steps", type=int, default=100)
    args = ap.parse_args(argv)
    case = CONFIGS[args.config]()
    w64, s64, e0, ms64 = run(case, "fp64", args.steps)
    wmx, smx, _, msmx = run(case, "mixed", args.steps)
    scale = np.max(np.abs(w64), axis=(1, 2, 3))
    err = (np.max(np.abs(wmx - w64), axis=(1, 2, 3)) / scale).tolist()
    out = {"config": args.config, "points": case.points, "steps": args.steps,
           "err_mixed_vs_fp64": dict(zip(["rho", "rho_u", "rho_v", "rho_w", "rho_E"], err)),
           "energy0": e0, "energy_fp64": s64["energy"], "energy_mixed": smx["energy"],
           "energy_drift_mixed_vs_fp64": (smx["energy"] - s64["energy"]) / abs(s64["energy"]),
           "energy_change_fp64": (s64["energy"] - e0) / abs(e0),
           "mass_drift_mixed_vs_fp64": (smx["mass"] - s64["mass"]) / abs(s64["mass"]),
           "t_fp64": s64["t"], "t_mixed": smx["t"],
           "ms_per_step_fp64": ms64, "ms_per_step_mixed": msmx,
           "weno_frac_fp64": s64["weno_frac"], "weno_frac_mixed": smx["weno_frac"]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
