#!/usr/bin/env python
"""Benchmark: grid-point RK3 steps per second of the FP64 solver.

Workload: the compressible turbulent channel, bulk Mach 1.5, Re_tau ~ 220,
256 x 128 x 128 points (6 pi h x 2h x 2 pi h, tanh-stretched y, isothermal
walls, constant mass flow), hybrid central-6 / WENO5 where the sensor
exceeds 0.2, 6th-order viscous terms, dt from CFL 0.8 every 10 steps.
Synthetic seeded initial state (laminar Poiseuille profile plus 10 %
smooth random velocity perturbations).

One step = one full RK3 step (3 RHS stages) of the whole grid.  The state
(168 MB) and the working set (~1.2 GB) are larger than the 129 MB L2, so no
L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun as independent replicas (the solver does not
shard across GPUs); value = all ranks' point-steps / the slowest rank's time.
The reference arm times the plain CPU oracle on the host cores.

Beside the FP64 line: the same workload in mixed precision (`mixed`), with
a thermally perfect gas (`thermally_perfect`), and a short continuous-
batching serving run for the p50/p99 batched step latency (`serving`).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK3 steps/s"
UNIT = "point-steps/s"

# FP64 work per interior point of one launch of each kernel as formulated
# (ncu, channel 256x128x128 hybrid: dadd + dmul + 2 dfma thread
# instructions / points for FLOPS; every FP64-pipe instruction for OPS).
# The FP64 unit issues one add, multiply or fused multiply-add per slot,
# so OPS against the slot rate is the pipe utilisation and FLOPS against
# 2 flop/slot the flop-rate fraction.
ALG_FLOPS = {"prims": 61.0, "grad": 81.0, "flux_x": 90.6, "flux_y": 92.1, "flux_z": 91.1, "visc": 252.7, "update": 20.0}
FP64_OPS = {"prims": 47.0, "grad": 64.0, "flux_x": 59.5, "flux_y": 60.5, "flux_z": 59.5, "visc": 170.4, "update": 15.0}
# DRAM bytes per interior point of one launch from the same ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); None where not captured.
DRAM_BYTES = {"prims": 92.1, "grad": 102.3, "flux_x": 89.7, "flux_y": 134.7, "flux_z": 134.7, "visc": 207.4, "update": 155.0}
# FP64 peak: 152 SMs x 2 DFMA/clk (4 flop) x 2070 MHz maximum SM clock.
FP64_PEAK_GFLOPS = 152 * 4 * 2.070
FP64_PEAK_GOPS = FP64_PEAK_GFLOPS / 2
# Mixed path: algorithmic HBM bytes per interior point of one launch
# (single-precision primitives and RHS, double-precision state; each field
# read or written once, halos not counted):
#   prims  w (40) -> rho, u, v, w, T, p, H, mu (32)
#   grad   u, v, w (12) -> div u, sensor test (8)
#   flux   rho, u, v, w, H, p, sensor (28) + RHS write (20), y and z also read it (20)
#   visc   u, v, w, T, div u, mu (24) + RHS read and write (40)
#   update w read/write (80), RHS (20), RK register read and write on 2 of 3 stages (26.7), u (4)
MIXED_BYTES = {"prims": 72, "grad": 20, "flux_x": 48, "flux_y": 68, "flux_z": 68, "visc": 64, "update": 130.7}
# DRAM bytes per interior point of one launch of the mixed kernels (ncu,
# same workload, captured with the current kernels; stage 0 of a step that
# recomputes dt): the traffic of the reported kernel.
MIXED_DRAM_BYTES = {"prims": 63.9, "visc": 65.3, "update": 110.6}
# Thermally perfect gas of the side measurement: a synthetic polynomial of
# the NASA 9-coefficient form, c_p/R = sum_{l=-2..4} a_l T^l (reference
# units of T), whose gamma falls from 1.45 at T = 0.5 through 1.40 at T = 1
# to 1.35 at T = 2, with the T^-2 and logarithmic T^-1 terms present.
TP_GAS = [0.05, -0.2, 3.2, 0.5, -0.06, 0.004, 0.0]


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-tp", action="store_true", help="skip the thermally perfect gas measurement")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the short serving run (p50/p99 batched step latency); 0 skips it")
    return ap.parse_args()


def workload():
    from paper_2304_05494_gb300 import workloads as W
    return W.channel()


def config_of(case):
    return {"workload": "compressible channel %dx%dx%d (6pi x 2 x 2pi, tanh y, M_b=1.5, Re_tau~220), "
                        "FP64 hybrid central-6/WENO5 (sensor>0.2), viscous-6, RK3, CFL 0.8 dt every 10"
                        % (case.nx, case.ny, case.nz),
            "points": case.points, "grid": [case.nx, case.ny, case.nz], "seed": 1235,
            "l2": "inputs larger than L2 (state 168 MB, working set ~1.2 GB > 129 MB L2); no flush"}


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(case, budget_s: float = 15.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    import numpy as np  # noqa: F401
    from oracle import oracle as O
    O.build()
    pr = O.Problem(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, y=case.y, mach=case.mach, re=case.re,
                   visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y, t_wall=case.t_wall,
                   force=case.force, weno_order=case.weno_order, threshold=case.threshold)
    t0 = time.perf_counter()
    O.step(pr, case.w0, 1, cfl=case.cfl, dt_every=case.dt_every)
    one = time.perf_counter() - t0
    steps = max(1, min(10, int(budget_s / max(one, 1e-3)) - 1))
    t0 = time.perf_counter()
    O.step(pr, case.w0, steps, cfl=case.cfl, dt_every=case.dt_every)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": case.points * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK3 step(s) of the full %dx%dx%d channel after 1 untimed step (%.1f s)"
                      % (steps, case.nx, case.ny, case.nz, el),
            "single_core": cpu_single_core()}


SINGLE_CORE_CODE = """
import json, os, sys, time
sys.path.insert(0, %r)
import bench
from oracle import oracle as O
case = bench.workload()
sub = 16
w = case.w0[:, :sub].copy()
pr = O.Problem(case.nx, case.ny, sub, case.lx, case.ly, case.lz * sub / case.nz, y=case.y, mach=case.mach,
               re=case.re, visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y, t_wall=case.t_wall,
               force=case.force, weno_order=case.weno_order, threshold=case.threshold)
t0 = time.perf_counter()
O.step(pr, w, 1, cfl=case.cfl, dt_every=case.dt_every)
el = time.perf_counter() - t0
print(json.dumps({"value": case.nx * case.ny * sub / el, "seconds": el}))
"""


def cpu_single_core():
    """The oracle on one host core (a fresh process with OMP_NUM_THREADS=1):
    one RK3 step of a 16-plane z-slab of the workload."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", SINGLE_CORE_CODE % ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    v = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": v["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "1 RK3 step of a 16-plane z-slab of the channel (%.1f s)" % v["seconds"]}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    import numpy as np
    case = workload()
    O.build()
    # bounded sample: a z-slab of nz/8 planes of the channel (same spacing),
    # so that one RK3 step of the oracle takes a second or so here
    nz = case.nz
    sub = max(4, nz // 8)
    w = np.ascontiguousarray(case.w0[:, :sub])
    lz = case.lz * sub / nz
    pr = O.Problem(case.nx, case.ny, sub, case.lx, case.ly, lz, y=case.y, mach=case.mach, re=case.re,
                   visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y, t_wall=case.t_wall,
                   force=case.force, weno_order=case.weno_order, threshold=case.threshold)
    st, dt = 0, 0.0
    for _ in range(args.warmup):
        w, st, dt = O.step(pr, w, 1, cfl=case.cfl, dt_every=case.dt_every, step0=st, dt0=dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w, st, dt = O.step(pr, w, 1, cfl=case.cfl, dt_every=case.dt_every, step0=st, dt0=dt)
    el = time.perf_counter() - t0
    pts = case.nx * case.ny * sub
    value = pts * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "%d-plane z-slab (%dx%dx%d, same spacing) of the channel, one RK3 step per bench step" % (
        sub, case.nx, case.ny, sub)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(case),
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value, "unit": UNIT},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def our_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2304_05494_gb300 import s2

    case = workload()
    stream = torch.cuda.Stream()
    sv = s2.Solver.from_case(case, stream=stream.cuda_stream, device=local)
    sv.set_state(case.w0)
    # warm-up (graph capture happens here)
    sv.step(args.warmup)
    sv.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    torch.cuda.synchronize()
    launches0 = sv.stats()["launches"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sv.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    st = sv.stats()
    launches = st["launches"] - launches0
    t_max = ms
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = case.points * args.steps * world / (t_max * 1e-3)

    # per-kernel device times (CUDA events on the solver's stream)
    prof = sv.profile(args.profile_steps)
    st2 = sv.stats()
    weno_frac = st2["weno_frac"]
    dom = max(((k, v) for k, v in prof.items() if k in ALG_FLOPS), key=lambda kv: kv[1][0])
    name, (kms, kl) = dom
    per_launch_ms = kms / max(kl, 1)
    flops = ALG_FLOPS[name] * case.points
    achieved = flops / (per_launch_ms * 1e-3) / 1e9
    ops = FP64_OPS[name] * case.points / (per_launch_ms * 1e-3) / 1e9
    traffic = DRAM_BYTES.get(name)
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": traffic * case.points if traffic is not None else None, "kernel": name,
                "peak_source": "FP64 pipe: 152 SM x 4 flop/clk x 2070 MHz (measured FMA loop: 1204 GFLOP/s)",
                "fp64_pipe_frac": ops / FP64_PEAK_GOPS,
                "per_launch_ms": per_launch_ms,
                "kernels_ms_per_step": {k: v[0] / args.profile_steps for k, v in prof.items() if v[1]}}

    # mixed precision: same workload, single-precision flux arithmetic
    mixed = None
    if not args.no_mixed:
        sm = s2.Solver.from_case(case, stream=stream.cuda_stream, device=local, precision="mixed")
        sm.set_state(case.w0)
        sm.step(args.warmup)
        sm.sync()
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        sm.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_m = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms_m], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_m = float(t.item())
        prof_m = sm.profile(args.profile_steps)
        domm = max(((k, v) for k, v in prof_m.items() if k in MIXED_BYTES), key=lambda kv: kv[1][0])
        mname, (mms, ml) = domm
        per_launch = mms / max(ml, 1)
        peak, src = hbm_peak_gbs()
        ach = MIXED_BYTES[mname] * case.points / (per_launch * 1e-3) / 1e9
        # every mixed kernel against the same HBM peak (algorithmic bytes)
        kfrac = {k: MIXED_BYTES[k] * case.points / (v[0] / v[1] * 1e-3) / 1e9 / peak
                 for k, v in prof_m.items() if k in MIXED_BYTES and v[1]}
        # error of the mixed path against the FP64 path after 10 steps from w0
        sm.set_state(case.w0)
        sm.set_clock(0.0, 0, 0.0)
        sm.step(10)
        wm = sm.get_state()
        sm.close()
        with s2.Solver.from_case(case, stream=stream.cuda_stream, device=local) as sd:
            sd.set_state(case.w0)
            sd.step(10)
            wd = sd.get_state()
        scale = np.max(np.abs(wd), axis=(1, 2, 3))
        err = (np.max(np.abs(wm - wd), axis=(1, 2, 3)) / scale).tolist()
        mixed = {"value": case.points * args.steps * world / (ms_m * 1e-3), "unit": UNIT,
                 "ms_per_step": ms_m / args.steps, "dtype": "f32 flux / f64 state",
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "traffic": (MIXED_DRAM_BYTES[mname] * case.points if mname in MIXED_DRAM_BYTES
                                          else None), "kernel": mname, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)",
                              "per_launch_ms": per_launch, "hbm_frac_per_kernel": kfrac,
                              "kernels_ms_per_step": {k: v[0] / args.profile_steps for k, v in prof_m.items() if v[1]}},
                 "err_vs_fp64_after_10_steps": err}

    # thermally perfect gas (Sec. 2: c_p(T) from a NASA-form polynomial):
    # the same workload and initial flow (its primitive fields, converted
    # with this gas's e(T) on the device), FP64 and mixed precision
    tp = None
    if not args.no_tp:
        tp = {"gas": "synthetic NASA 9-coefficient form c_p/R = sum a_l T^l, a_-2..a_4 = %s "
                     "(gamma 1.45 / 1.40 / 1.35 at T = 0.5 / 1 / 2)" % TP_GAS}
        for prec in ("fp64", "mixed"):
            stp = s2.Solver.from_case(case, stream=stream.cuda_stream, device=local, precision=prec,
                                      cp_coeffs=TP_GAS)
            stp.set_primitives(case.prim0)
            stp.step(args.warmup)
            stp.sync()
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            stp.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            ms_t = e0.elapsed_time(e1)
            if world > 1:
                t = torch.tensor([ms_t], device="cuda", dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ms_t = float(t.item())
            prof_t = stp.profile(args.profile_steps)
            ok = stp.stats()["status"] == 0
            stp.close()
            tp[prec] = {"value": case.points * args.steps * world / (ms_t * 1e-3), "unit": UNIT,
                        "ms_per_step": ms_t / args.steps, "status_ok": ok,
                        "kernels_ms_per_step": {k: v[0] / args.profile_steps for k, v in prof_t.items() if v[1]}}

    # batched step latency: a short continuous-batching serving run (mixed
    # precision, Poisson arrivals at 80 % of the measured capacity of a full
    # batch, boxes of 32^3 .. 128^3, 50 .. 200 steps each)
    serving = None
    if args.serve_requests > 0 and world == 1:
        from paper_2304_05494_gb300 import serve
        cap = serve.capacity("mixed")
        reqs = serve.make_requests(args.serve_requests, steps=(50, 200), precisions=("mixed",))
        rate = 0.8 * cap / float(np.mean([r.points * r.steps for r in reqs]))
        serve.poisson_arrivals(reqs, rate)
        so = serve.Server(max_slots=64, steps_per_tick=10).run(reqs)
        serving = {"requests": so["requests"], "done": so["done"], "precision": "mixed", "load": 0.8,
                   "capacity": cap, "throughput": so["throughput"], "unit": UNIT,
                   "p50_step_latency_ms": so["p50_step_latency_ms"],
                   "p99_step_latency_ms": so["p99_step_latency_ms"],
                   "p50_queue_s": so["p50_queue_s"], "p99_queue_s": so["p99_queue_s"],
                   "workload": "Taylor-Green or seeded decaying turbulence boxes {32,48,64,96,128}^3, "
                               "M in [0.1, 0.8], Re in [400, 3200], 50-200 RK3 steps"}

    # end to end through the C ABI with host buffers: H2D of the step's
    # input state, one step, D2H of the result, every step
    pinned_in = torch.from_numpy(case.w0).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    win = pinned_in.numpy()
    wout = pinned_out.numpy()
    sv.set_state(win)
    sv.step(1)
    sv.get_state(wout)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sv.set_state(win)
        sv.step(1)
        sv.get_state(wout)
    t_e2e = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = float(t.item())
    nbytes = case.w0.nbytes
    e2e = {"value": case.points * args.e2e_steps * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    finite = bool(np.isfinite(wout).all())
    sv.close()

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(config_of(case), parallelism="replicas" if world > 1 else "single"),
               "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "mixed": mixed,
               "thermally_perfect": tp, "serving": serving, "weno_frac": weno_frac, "state_finite": finite}
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(case)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
