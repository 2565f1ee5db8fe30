#!/usr/bin/env python
"""Benchmark: grid-point RK3 steps per second of the solver.

Headline workload: the large compressible turbulent channel, bulk Mach 1.5,
Re_tau ~ 550, 1024 x 256 x 512 points (134M; 6 pi h x 2h x 2 pi h,
tanh-stretched y, first wall cell at dy+ = 0.7, isothermal walls, constant
mass flow), hybrid central-6 / WENO5 where the sensor exceeds 0.2,
6th-order viscous terms, dt from CFL 0.8 every 10 steps, in double
precision (`value`) and in mixed precision (`mixed`: single-precision
flux, WENO and viscous arithmetic, double-precision state and RK
accumulation).  Synthetic seeded initial state (laminar Poiseuille profile
plus 10 % smooth random velocity perturbations).

One step = one full RK3 step (3 RHS stages) of the whole grid.  The state
(5.4 GB) and the working set (tens of GB) are far larger than the 129 MB
L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun as independent replicas (the solver does not
shard across GPUs); value = all ranks' point-steps / the slowest rank's time.
The reference arm times the plain CPU oracle on the host cores.

Beside the headline: the 256 x 128 x 128 channel (Re_tau ~ 220) in both
precisions (`channel256`), the same with a thermally perfect gas
(`thermally_perfect`), the work-list batch against the member-branch graph
on many small boxes (`batching`), and a continuous-batching serving run of
the serving workload (256 requests) for the p50/p99 batched step latency
(`serving`).  The last keys of the line repeat the mixed-precision figures.
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

# Algorithmic double-precision operations per interior point of one launch
# of each kernel class: the CPU oracle's operation tally (oracle/tally.py;
# adds, multiplies, divides, square roots and pow/log/exp, one flop each)
# of the part of the method that the kernel computes, for the benchmark
# scheme (central 6, WENO5, viscous 6, calorically perfect gas).
# tests/test_oracle_tally.py checks them against a fresh tally.
#   prims   primitive recovery (14) and H, c (11)
#   grad    nine velocity gradients, divergence and shock sensor
#   visc    viscous and heat-flux terms, given the velocity gradients
#   update  RK3 update, 5 per field
ALG_FLOPS = {"prims": 25.0, "grad": 105.0, "visc": 383.0, "update": 25.0}
ALG_FLOPS_VISC_GRAD = 90.0            # the nine velocity gradients the viscous terms use
ALG_FLOPS_CENTRAL_INTERFACE = 226.0   # one split-form interface flux (5 fields)
ALG_FLOPS_WENO_INTERFACE = 1760.0     # one characteristic WENO5 interface flux
ALG_FLOPS_FLUX_DIFFERENCE = 47.0 / 3  # flux difference per point and direction
# Double-precision issue peak of the FP64 unit: 152 SMs x 2 DFMA per clock
# (4 flop) at the 2070 MHz maximum SM clock.
FP64_PEAK_GFLOPS = 152 * 4 * 2.070
# DRAM bytes per interior point of one launch of the FP64 viscous kernel
# (ncu dram__bytes_read.sum + dram__bytes_write.sum, 256 x 128 x 128
# channel, scaled by the points of a launch; profiles/channel256x128x128_fp64_visc_full.md).
FP64_DRAM_BYTES = {"visc": 207.8}
# Mixed path: algorithmic HBM bytes per interior point of one launch
# (single-precision primitives and RHS, double-precision state; each field
# read or written once, halos not counted):
#   prims  w (40) -> rho, u, v, w, T, p, H, mu (32)
#   grad   u, v, w (12) -> div u, sensor test (8)
#   flux   rho, u, v, w, H, p, sensor (28) + RHS write (20), y and z also read it (20)
#   visc   u, v, w, T, div u, mu (24) + RHS read and write (40)
#   update w read/write (80), RHS (20), RK register read and write on 2 of 3 stages (26.7), u (4)
MIXED_BYTES = {"prims": 72, "grad": 20, "flux_x": 48, "flux_y": 68, "flux_z": 68, "visc": 64, "update": 130.7}
# The method's algorithmic traffic per point and RK3 step: per stage read
# and write the state and the RK register, 4 x 40 B.
METHOD_BYTES_PER_POINT_STEP = 480.0
# DRAM bytes per interior point of one launch of the mixed kernels (ncu,
# 256 x 128 x 128 channel, first stage; profiles/channel256x128x128_mixed_kernels_full.md,
# the viscous pass profiles/channel1024x256x512_launch_list.md).
MIXED_DRAM_BYTES = {"prims": 63.9, "visc": 65.5, "update": 110.1}
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
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--err-steps", type=int, default=10,
                    help="steps of the mixed-vs-FP64 error measurement on the headline workload")
    ap.add_argument("--no-side", action="store_true", help="skip the 256x128x128 channel and thermally perfect legs")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving run (p50/p99 batched step latency); 0 skips it")
    ap.add_argument("--small", action="store_true", help="headline on the 256x128x128 channel (quick checks)")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batching comparison")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="mixed leg with the default launch knobs instead of the autotuner's")
    return ap.parse_args()


def workload(small: bool = False):
    from paper_2304_05494_gb300 import workloads as W
    return W.channel() if small else W.channel_big()


def config_of(case):
    retau = 550 if case.nx == 1024 else 220
    return {"workload": "compressible channel %dx%dx%d (6pi x 2 x 2pi, tanh y, M_b=1.5, Re_tau~%d), "
                        "hybrid central-6/WENO5 (sensor>0.2), viscous-6, RK3, CFL 0.8 dt every 10; "
                        "value FP64, mixed = f32 flux/f64 state" % (case.nx, case.ny, case.nz, retau),
            "points": case.points, "grid": [case.nx, case.ny, case.nz], "seed": case_seed(case),
            "l2": "inputs larger than L2 (state %.1f GB > 129 MB L2); no flush" % (case.w0.nbytes / 1e9)}


def case_seed(case):
    return 1234 + (3 if case.nx == 1024 else 1)


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


def _problem(O, case, nz=None):
    sub = case.nz if nz is None else nz
    return O.Problem(case.nx, case.ny, sub, case.lx, case.ly, case.lz * sub / case.nz, y=case.y, mach=case.mach,
                     re=case.re, visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y,
                     t_wall=case.t_wall, force=case.force, weno_order=case.weno_order, threshold=case.threshold)


def slab_planes(case) -> int:
    """z-slab of the workload that one oracle RK3 step covers in a second or
    two on a many-core host (8 planes of 1024 x 256, or 16 of 256 x 128)."""
    return max(4, min(case.nz, (2 << 20) // (case.nx * case.ny)))


def cpu_baseline(case, budget_s: float = 15.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload: RK3
    steps of a z-slab (same grid spacing, same flow) on all host cores."""
    import numpy as np
    from oracle import oracle as O
    O.build()
    sub = slab_planes(case)
    w = np.ascontiguousarray(case.w0[:, :sub])
    pr = _problem(O, case, sub)
    t0 = time.perf_counter()
    w1, st, dt = O.step(pr, w, 1, cfl=case.cfl, dt_every=case.dt_every)
    one = time.perf_counter() - t0
    steps = max(1, min(10, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    O.step(pr, w1, steps, cfl=case.cfl, dt_every=case.dt_every, step0=st, dt0=dt)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    pts = case.nx * case.ny * sub
    return {"value": pts * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK3 step(s) of a %d-plane z-slab (%dx%dx%d, same spacing) of the workload after 1 "
                      "untimed step (%.1f s)" % (steps, sub, case.nx, case.ny, sub, el),
            "single_core": cpu_single_core(case)}


SINGLE_CORE_CODE = """
import json, os, sys, time
sys.path.insert(0, %r)
import bench
import numpy as np
from oracle import oracle as O
case = bench.workload(%r)
sub = 2
w = np.ascontiguousarray(case.w0[:, :sub])
pr = bench._problem(O, case, sub)
t0 = time.perf_counter()
O.step(pr, w, 1, cfl=case.cfl, dt_every=case.dt_every)
el = time.perf_counter() - t0
print(json.dumps({"value": case.nx * case.ny * sub / el, "seconds": el, "planes": sub}))
"""


def cpu_single_core(case):
    """The oracle on one host core (a fresh process with OMP_NUM_THREADS=1):
    one RK3 step of a 2-plane z-slab of the workload."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    small = case.nx != 1024
    r = subprocess.run([sys.executable, "-c", SINGLE_CORE_CODE % (ROOT, small)], env=env, capture_output=True,
                       text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    v = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": v["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "1 RK3 step of a %d-plane z-slab of the workload (%.1f s)" % (v["planes"], v["seconds"])}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    case = workload(args.small)
    O.build()
    # bounded sample: a z-slab of the workload (same spacing, same flow) so
    # that one RK3 step of the oracle takes a second or so here
    sub = slab_planes(case)
    w = np.ascontiguousarray(case.w0[:, :sub])
    pr = _problem(O, case, sub)
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
    sample = "%d-plane z-slab (%dx%dx%d, same spacing) of the workload, one RK3 step per bench step" % (
        sub, case.nx, case.ny, sub)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(case),
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value, "unit": UNIT},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


class Timer:
    """Device time of a region on one stream (CUDA events), max over ranks.

    The ranks are independent replicas: the only collectives are the
    barriers around the timed region and the max of the times (on the
    device for NCCL, on the host for gloo)."""

    def __init__(self, torch, dist, world, stream, device="cuda"):
        self.torch, self.dist, self.world, self.stream, self.device = torch, dist, world, stream, device

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def run(self, fn):
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        self.barrier()
        torch.cuda.synchronize()
        e0.record(self.stream)
        fn()
        e1.record(self.stream)
        torch.cuda.synchronize()
        self.barrier()
        return self.max(e0.elapsed_time(e1))

    def max(self, v):
        if self.world > 1:
            t = self.torch.tensor([v], device=self.device, dtype=self.torch.float64)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
            v = float(t.item())
        return v


def whole_job_rate(points, steps, world, ms):
    """Point-steps per second of the whole job: every rank advances its own
    replica of `points` points by `steps` steps; `ms` is the slowest rank's
    time."""
    return points * steps * world / (ms * 1e-3)


def per_launch(prof, name):
    ms, n = prof.get(name, (0.0, 0))
    return ms / n if n else None


def fp64_roofline(case, prof, steps, weno_frac, step_ms, fma_gflops):
    """FP64 path: bound by the double-precision unit.  achieved = the
    oracle-tallied flops of the dominant kernel class per launch / its mean
    launch time (CUDA events on the solver's stream); the whole step's
    tallied flops / step time beside it."""
    n = case.points
    flux_pp = {d: ALG_FLOPS_CENTRAL_INTERFACE * (nd + 1) / nd + ALG_FLOPS_FLUX_DIFFERENCE
               for d, nd in (("flux_x", case.nx), ("flux_y", case.ny), ("flux_z", case.nz))}
    alg = dict(ALG_FLOPS, **flux_pp)
    # WENO corrections: flagged interfaces (weno_frac x 3N per stage) x the
    # WENO flux minus the central flux it replaces
    weno_pl = weno_frac * 3 * n * (ALG_FLOPS_WENO_INTERFACE - ALG_FLOPS_CENTRAL_INTERFACE) / 3
    kernels = {k: v for k, v in prof.items() if v[1] and (k in alg or k == "weno")}
    name = max(kernels, key=lambda k: kernels[k][0])
    pl = per_launch(prof, name)
    flops = (weno_pl if name == "weno" else alg[name] * n)
    achieved = flops / (pl * 1e-3) / 1e9
    per_kernel = {}
    for k in kernels:
        f = weno_pl if k == "weno" else alg[k] * n
        per_kernel[k] = round(f / (per_launch(prof, k) * 1e-3) / 1e9 / FP64_PEAK_GFLOPS, 3)
    step_flops = 3 * (sum(alg[k] for k in ("prims", "grad", "visc", "update", "flux_x", "flux_y", "flux_z"))
                      + weno_frac * 3 * (ALG_FLOPS_WENO_INTERFACE - ALG_FLOPS_CENTRAL_INTERFACE)) * n
    traffic = FP64_DRAM_BYTES.get(name)
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic * n if traffic else None, "kernel": name,
            "per_launch_ms": pl,
            "peak_source": "152 SM x 2 DFMA/clk x 2070 MHz (FP64 unit issue rate); FMA loop measured live: "
                           "%.0f GFLOP/s" % fma_gflops,
            "frac_of_fma_measured": achieved / fma_gflops,
            "flops_source": "oracle operation tally (oracle/tally.py)",
            "step_frac": step_flops / (step_ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
            "frac_per_kernel": per_kernel}


def mixed_roofline(case, prof, step_ms):
    """Mixed path: HBM.  The method's 480 B per point-step against the
    step time, and per kernel the algorithmic bytes of its launch."""
    n = case.points
    peak, src = hbm_peak_gbs()
    kernels = {k: v for k, v in prof.items() if v[1] and k in MIXED_BYTES}
    name = max(kernels, key=lambda k: kernels[k][0])
    pl = per_launch(prof, name)
    ach = MIXED_BYTES[name] * n / (pl * 1e-3) / 1e9
    kfrac = {k: round(MIXED_BYTES[k] * n / (per_launch(prof, k) * 1e-3) / 1e9 / peak, 3) for k in kernels}
    step_gbs = METHOD_BYTES_PER_POINT_STEP * n / (step_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": MIXED_DRAM_BYTES[name] * n if name in MIXED_DRAM_BYTES else None, "kernel": name,
            "per_launch_ms": pl, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)",
            "step_frac": step_gbs / peak, "step_bytes_per_point": METHOD_BYTES_PER_POINT_STEP,
            "frac_per_kernel": kfrac}


def batch_leg(s2, steps=10):
    """Many small boxes batched: ms per batch step of the work-list batch
    (one launch per kernel for all boxes) and of the member-branch graph,
    for 64 Taylor-Green boxes of 24^3 (hybrid WENO5) and for one box of each
    serving size 32^3 .. 128^3, in mixed precision."""
    import time
    from paper_2304_05494_gb300 import workloads as W
    out = {}
    for name, sizes in (("64x24^3", [24] * 64), ("32^3..128^3", [32, 48, 64, 96, 128])):
        cases = [W.taylor_green(n, mach=0.3, seed=10 + i) for i, n in enumerate(sizes)]
        for c in cases:
            c.weno_order, c.threshold = 5, 0.2
        res = {}
        for mode in ("branches", "worklist"):
            solvers = []
            for c in cases:
                sv = s2.Solver.from_case(c, precision="mixed")
                sv.set_state(c.w0)
                solvers.append(sv)
            with s2.Batch(solvers, mode=mode) as b:
                b.step(2)
                b.sync()
                best = 1e9
                for _ in range(3):
                    t0 = time.perf_counter()
                    b.step(steps)
                    b.sync()
                    best = min(best, time.perf_counter() - t0)
                res[mode] = {"ms_per_step": best / steps * 1e3, "launches_per_step": b.launches_per_step}
            for sv in solvers:
                sv.close()
        res["speedup"] = res["branches"]["ms_per_step"] / res["worklist"]["ms_per_step"]
        out[name] = res
    return out


def ms_per_step(prof, steps):
    return {k: round(v[0] / steps, 4) for k, v in prof.items() if v[1]}


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
    from paper_2304_05494_gb300 import autotune, s2

    case = workload(args.small)
    stream = torch.cuda.Stream()
    T = Timer(torch, dist, world, stream)
    fma = s2.s2_fma_rate("fp64", local)

    # ---- headline: FP64 --------------------------------------------------
    sv = s2.Solver.from_case(case, stream=stream.cuda_stream, device=local)
    sv.set_state(case.w0)
    sv.step(args.warmup)  # graph capture happens here
    sv.sync()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.4)
    launches0 = sv.stats()["launches"]
    t_max = T.run(lambda: sv.step(args.steps))
    clk = clocks.stop()
    launches = sv.stats()["launches"] - launches0
    value = whole_job_rate(case.points, args.steps, world, t_max)
    prof = sv.profile(args.profile_steps)
    weno_frac = sv.stats()["weno_frac"]
    roofline = fp64_roofline(case, prof, args.profile_steps, weno_frac, t_max / args.steps, fma)
    roofline["kernels_ms_per_step"] = ms_per_step(prof, args.profile_steps)

    # end to end through the C ABI with host buffers: every step the H2D
    # copy of its input state from pinned memory, one RK3 step, the D2H copy
    # of its result (s2_stream_states: the copies of the next input and the
    # previous result overlap the step)
    pinned_in = torch.from_numpy(case.w0).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    win, wout = pinned_in.numpy(), pinned_out.numpy()
    sv.stream_states(win, wout, 1, count=1)  # first call: staging buffers
    T.barrier()
    t0 = time.perf_counter()
    sv.stream_states(win, wout, 1, count=args.e2e_steps)
    t_e2e = T.max(time.perf_counter() - t0)
    e2e = {"value": whole_job_rate(case.points, args.e2e_steps, world, t_e2e * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": case.w0.nbytes, "d2h_bytes_per_step": case.w0.nbytes}
    finite = bool(np.isfinite(wout[:, ::64]).all())
    del pinned_in, pinned_out, win, wout

    # ---- mixed precision, same workload ----------------------------------
    sm = s2.Solver.from_case(case, stream=stream.cuda_stream, device=local, precision="mixed")
    # launch knobs from the project's autotuner for this grid (cached per
    # grid, precision, WENO order and GPU; a miss tunes for a few seconds,
    # outside the timed region, and restores the state and the clock)
    tuning = None
    if args.tune:
        tuning = autotune.tuning_for(sm, case.w0, (case.nx, case.ny, case.nz), "mixed", case.weno_order, steps=2)
    sm.set_state(case.w0)
    sm.step(args.warmup)
    sm.sync()
    ms_m = T.run(lambda: sm.step(args.steps))
    prof_m = sm.profile(args.profile_steps)
    mroof = mixed_roofline(case, prof_m, ms_m / args.steps)
    mroof["kernels_ms_per_step"] = ms_per_step(prof_m, args.profile_steps)
    # error of the mixed path against the FP64 path after err_steps steps
    # from the same state, per conserved field (field-normalised), and the
    # relative difference of the total energy
    err = energy_drift = None
    if args.err_steps > 0:
        for s in (sm, sv):
            s.set_state(case.w0)
            s.set_clock(0.0, 0, 0.0)
            s.step(args.err_steps)
        e_m, e_d = sm.stats()["energy"], sv.stats()["energy"]
        wm = sm.get_state()
        wd = sv.get_state()
        err = [float(np.max(np.abs(wm[f] - wd[f])) / np.max(np.abs(wd[f]))) for f in range(5)]
        energy_drift = (e_m - e_d) / abs(e_d)
        del wm, wd
    sm.close()
    sv.close()
    mixed = {"value": whole_job_rate(case.points, args.steps, world, ms_m), "unit": UNIT,
             "ms_per_step": ms_m / args.steps, "dtype": "f32 flux / f64 state", "tuning": tuning, "roofline": mroof,
             "err_vs_fp64": err, "energy_rel_diff_vs_fp64": energy_drift, "err_steps": args.err_steps}

    # ---- side legs on the 256 x 128 x 128 channel ------------------------
    side = tp = None
    if not args.no_side and not args.small:
        side = {"workload": "compressible channel 256x128x128, Re_tau~220, same scheme"}
        c2 = workload(True)
        for prec in ("fp64", "mixed"):
            s = s2.Solver.from_case(c2, stream=stream.cuda_stream, device=local, precision=prec)
            s.set_state(c2.w0)
            s.step(args.warmup)
            s.sync()
            ms = T.run(lambda: s.step(args.steps))
            s.close()
            side[prec] = {"value": whole_job_rate(c2.points, args.steps, world, ms), "ms_per_step": ms / args.steps}
        # thermally perfect gas (Sec. 2: c_p(T) from a NASA-form polynomial):
        # the same flow, converted with this gas's e(T) on the device
        tp = {"gas": "synthetic NASA 9-coefficient form, a_-2..a_4 = %s" % TP_GAS, "workload": "channel 256x128x128"}
        for prec in ("fp64", "mixed"):
            s = s2.Solver.from_case(c2, stream=stream.cuda_stream, device=local, precision=prec, cp_coeffs=TP_GAS)
            s.set_primitives(c2.prim0)
            s.step(args.warmup)
            s.sync()
            ms = T.run(lambda: s.step(args.steps))
            ok = s.stats()["status"] == 0
            s.close()
            tp[prec] = {"value": whole_job_rate(c2.points, args.steps, world, ms), "ms_per_step": ms / args.steps,
                        "status_ok": ok}

    # ---- batching: work-list batch against member branches -------------
    batching = None
    if args.batch and world == 1:
        batching = batch_leg(s2)

    # ---- serving: continuous batching at 80 % of capacity ----------------
    serving = None
    if args.serve_requests > 0 and world == 1:
        from paper_2304_05494_gb300 import serve
        cap = serve.capacity("mixed")
        reqs = serve.make_requests(args.serve_requests, steps=(100, 1000), precisions=("mixed",))
        rate = 0.8 * cap / float(np.mean([r.points * r.steps for r in reqs]))
        serve.poisson_arrivals(reqs, rate)
        so = serve.Server(max_slots=64, steps_per_tick=10).run(reqs)
        serving = {"requests": so["requests"], "done": so["done"], "precision": "mixed", "load": 0.8,
                   "capacity": cap, "throughput": so["throughput"], "unit": UNIT,
                   "p50_step_latency_ms": so["p50_step_latency_ms"],
                   "p99_step_latency_ms": so["p99_step_latency_ms"],
                   "p50_queue_s": so["p50_queue_s"], "p99_queue_s": so["p99_queue_s"],
                   "wall_s": round(so["wall_s"], 2), "ticks": so["ticks"],
                   "host_s": {k: round(v, 3) for k, v in so["host_s"].items()},
                   "workload": "Taylor-Green or seeded decaying turbulence boxes {32,48,64,96,128}^3, "
                               "M in [0.1, 0.8], Re in [400, 3200], 100-1000 RK3 steps, Poisson arrivals"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(config_of(case), parallelism="replicas" if world > 1 else "single"),
               "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
               "weno_frac": weno_frac, "state_finite": finite, "channel256": side, "thermally_perfect": tp,
               "batching": batching, "serving": serving, "mixed": mixed}
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(case)
        # the mixed-precision headline figures again, last on the line
        out["mixed_value"] = mixed["value"]
        out["mixed_ms_per_step"] = mixed["ms_per_step"]
        out["mixed_step_hbm_frac"] = mroof["step_frac"]
        out["mixed_roofline_frac"] = mroof["frac"]
        out["mixed_err_vs_fp64"] = err
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
