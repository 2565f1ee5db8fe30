"""The single-GPU performance studies of the paper's Sec. 4.1, run on GB300.

Three sweeps, one JSON line per configuration:

  orders  the order of accuracy on the paper's grid 420 x 250 x 320
          (compressible channel): central C2/C4/C6/C8 with viscous terms of
          the same order, sensor off; WENO W1/W3/W5/W7 at every interface
          (central and viscous order 6).  Reports the time per RK3 step and
          the euler_y (y-direction flux, plus its WENO corrections) time
          per launch -- the quantities of the paper's order-of-accuracy
          study.
  grid    grind time (ns per grid-point RK3 step) against the number of
          points, from ~0.26 M to ~134 M points (Taylor-Green box n^3,
          n = 64 ... 512, doubling the point count), central and WENO at
          every interface -- the paper's grid-size study, which finds GPUs
          need ~2 M points to fill up.
  weno    the fraction of WENO interfaces: an isotropic turbulent box
          (256^3, M_t = 0.6, WENO5) with the sensor threshold swept from
          "never" to "always"; reports the flagged fraction and the time
          per step -- the paper's WENO-activation study.  Flagged
          interfaces are compacted into lists here, so the cost should grow
          linearly with the fraction instead of through thread divergence.

  python -m paper_2304_05494_gb300.sweeps orders|grid|weno [--precision fp64 mixed]

Times are CUDA-event device times on the solver's stream over a number of
steps chosen to last ~0.3 s (four in the WENO-activation sweep, where the
flow must evolve alike in both precisions), after two warm-up steps;
per-kernel times come from s2_profile (CUDA events per kernel class).
"""
from __future__ import annotations

import argparse
import json

from . import workloads as W

PAPER_GRID = (420, 250, 320)


def timed(case, precision: str, target_s: float = 0.3, steps: int = 0, **kw) -> dict:
    import torch
    from . import s2
    stream = torch.cuda.Stream()
    with s2.Solver.from_case(case, stream=stream.cuda_stream, precision=precision, **kw) as sv:
        sv.set_state(case.w0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sv.step(2)  # graph capture and warm-up
        sv.sync()
        frac0 = sv.stats()["weno_frac"]
        if steps <= 0:
            e0.record(stream)
            sv.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            one = e0.elapsed_time(e1)
            steps = max(3, min(400, int(target_s * 1e3 / max(one, 1e-3))))
        e0.record(stream)
        sv.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = sv.profile(2)
        st = sv.stats()
    per_step = {k: v[0] / 2 for k, v in prof.items() if v[1]}
    per_launch = {k: v[0] / v[1] for k, v in prof.items() if v[1]}
    return {"points": case.points, "steps": steps, "ms_per_step": ms,
            "point_steps_per_s": case.points / (ms * 1e-3), "grind_ns": ms * 1e6 / case.points,
            "weno_frac": st["weno_frac"], "weno_frac_start": frac0, "status": st["status"],
            "kernels_ms_per_step": per_step,
            "kernels_ms_per_launch": per_launch}


def orders(precisions):
    case = W.channel(*PAPER_GRID)
    for precision in precisions:
        for order in (2, 4, 6, 8):
            r = timed(case, precision, weno_order=0, central_order=order, visc_order=order)
            print(json.dumps({"sweep": "orders", "scheme": "C%d/V%d" % (order, order), "precision": precision,
                              "grid": list(PAPER_GRID), "ms_per_step": r["ms_per_step"],
                              "point_steps_per_s": r["point_steps_per_s"],
                              "euler_y_ms_per_launch": r["kernels_ms_per_launch"].get("flux_y"),
                              "kernels_ms_per_step": r["kernels_ms_per_step"]}), flush=True)
        for wo in (1, 3, 5, 7):
            r = timed(case, precision, weno_order=wo, threshold=-1.0)
            weno_y = r["kernels_ms_per_launch"].get("weno", 0.0)  # three directions per launch group
            print(json.dumps({"sweep": "orders", "scheme": "W%d (everywhere)" % wo, "precision": precision,
                              "grid": list(PAPER_GRID), "ms_per_step": r["ms_per_step"],
                              "point_steps_per_s": r["point_steps_per_s"],
                              "euler_y_ms_per_launch": r["kernels_ms_per_launch"].get("flux_y"),
                              "weno_ms_per_launch_mean": weno_y, "weno_frac": r["weno_frac"],
                              "kernels_ms_per_step": r["kernels_ms_per_step"]}), flush=True)


def grid(precisions):
    for n in (64, 80, 101, 128, 161, 203, 256, 322, 406, 512):
        case = W.taylor_green(n)
        for precision in precisions:
            for scheme, kw in (("central", dict(weno_order=0)), ("weno5 everywhere", dict(weno_order=5, threshold=-1.0))):
                r = timed(case, precision, **kw)
                print(json.dumps({"sweep": "grid", "n": n, "points": case.points, "scheme": scheme,
                                  "precision": precision, "grind_ns": r["grind_ns"],
                                  "ms_per_step": r["ms_per_step"], "point_steps_per_s": r["point_steps_per_s"]}),
                      flush=True)
        del case


def weno(precisions):
    case = W.isotropic(256, mach_t=0.6, weno_order=5)
    for precision in precisions:
        for thr in (1.01, 0.8, 0.6, 0.4, 0.3, 0.2, 0.1, 0.05, 0.02, -1.0):
            # the same few steps in both precisions, so that the flow (and so
            # the flagged fraction) evolves alike
            r = timed(case, precision, steps=4, threshold=thr)
            print(json.dumps({"sweep": "weno", "grid": [case.nx, case.ny, case.nz], "threshold": thr,
                              "precision": precision, "weno_frac_start": r["weno_frac_start"],
                              "weno_frac": r["weno_frac"], "ms_per_step": r["ms_per_step"],
                              "weno_ms_per_step": r["kernels_ms_per_step"].get("weno", 0.0),
                              "point_steps_per_s": r["point_steps_per_s"]}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("sweep", choices=["orders", "grid", "weno"])
    ap.add_argument("--precision", nargs="+", default=["fp64", "mixed"], choices=["fp64", "mixed"])
    args = ap.parse_args(argv)
    {"orders": orders, "grid": grid, "weno": weno}[args.sweep](args.precision)


if __name__ == "__main__":
    main()
