"""Continuous-batching serving loop for ensembles of independent box solves.

Requests (periodic boxes: Taylor-Green or seeded decaying turbulence, of
different sizes, Mach and Reynolds numbers, step counts and precisions)
arrive over time.  The server admits a request as soon as a slot and enough
device memory are free, keeps its state resident on the GPU, and advances
all admitted boxes together: each tick is one s2_batch_step, a single CUDA
graph launch whose branches are the members' RK3 steps, so boxes too small
to fill the GPU alone fill it together.  Requests that arrive while others
are running join at the next tick; finished ones leave and free their slot
and memory.  Each box's arithmetic is independent of the others (no shared
buffers, deterministic kernels), so a result is the same alone and in the
mix.

Reported: throughput (point-steps/s over the run), p50/p99 of the per-step
latency seen by requests (tick time / steps per tick), queueing delay.  A
request whose solve fails on the device (e.g. a non-positive density,
S2_ENONFINITE) is retired with that status and a request its client
cancels is retired at the next tick; the others continue unaffected.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import workloads as W

SIZES = (32, 48, 64, 96, 128)
# device bytes per grid point (state, registers, padded primitives,
# gradients, hybrid-scheme lists), measured from s2_create's allocations
BYTES_PER_POINT = {"fp64": 560, "mixed": 294}


@dataclass
class Request:
    rid: int
    n: int
    mach: float
    re: float
    steps: int
    kind: str          # "tgv" or "turb"
    precision: str     # "fp64" or "mixed"
    seed: int
    arrival: float = 0.0
    cancel_after: Optional[int] = None  # the client cancels after this many steps (None: never)
    corrupt: bool = False               # fault injection: a negative density in the initial state
    # filled by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    status: str = "pending"             # "done", "cancelled" or "failed: <error>"
    result: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def points(self) -> int:
        return self.n ** 3


def make_requests(count: int, seed: int = 4321, sizes=SIZES, steps=(100, 1000), precisions=("mixed",),
                  mach=(0.1, 0.8), re=(400.0, 3200.0), kinds=("tgv", "turb")) -> List[Request]:
    """The serving workload: sizes, Mach, Re, step counts and case kinds
    drawn uniformly from the given ranges (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append(Request(rid=i, n=int(rng.choice(sizes)), mach=float(rng.uniform(*mach)),
                           re=float(rng.uniform(*re)), steps=int(rng.integers(steps[0], steps[1] + 1)),
                           kind=str(rng.choice(kinds)), precision=str(rng.choice(precisions)),
                           seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out


def poisson_arrivals(reqs: List[Request], rate: float, seed: int = 99) -> None:
    """Exponential inter-arrival times with the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    for r in reqs:
        r.arrival = t
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0


def initial_case(req: Request) -> W.Case:
    if req.kind == "tgv":
        c = W.taylor_green(req.n, mach=req.mach, re=req.re, seed=req.seed)
    else:
        c = W.isotropic(req.n, mach_t=req.mach, re_lambda=0.0, seed=req.seed, weno_order=5)
        c.re = req.re
    c.weno_order = 5
    c.threshold = 0.2
    c.cfl = 0.8
    c.dt_every = 10
    if req.corrupt:
        c.w0 = c.w0.copy()
        c.w0[0, req.n // 2, req.n // 3, req.n // 4] = -1.0
    return c


class Server:
    def __init__(self, hbm_budget: Optional[float] = None, max_slots: int = 64, steps_per_tick: int = 10,
                 keep_results: bool = False, stream=None):
        import torch
        from . import s2
        self.s2 = s2
        self.torch = torch
        if hbm_budget is None:
            free, total = torch.cuda.mem_get_info()
            hbm_budget = 0.8 * free
        self.budget = hbm_budget
        self.max_slots = max_slots
        self.k = steps_per_tick
        self.keep = keep_results
        self.stream = stream

    @staticmethod
    def _left(a) -> int:
        """Steps the tick may take for one active entry (request, solver, remaining)."""
        r, left = a[0], a[2]
        if r.cancel_after is not None:
            left = min(left, max(r.cancel_after - (r.steps - a[2]), 1))
        return left

    def _bytes(self, req: Request) -> float:
        n = req.n
        return BYTES_PER_POINT[req.precision] * (n + 8) ** 3

    def run(self, reqs: List[Request], log=None) -> dict:
        """Serve the requests (arrival times relative to the call).  A request
        that has arrived has its initial field built on a host thread while
        the GPU works on the running batch; it is admitted (solver created,
        state copied in) at the next tick with a free slot and memory."""
        from concurrent.futures import ThreadPoolExecutor
        s2 = self.s2
        pending = sorted(reqs, key=lambda r: r.arrival)
        prep = ThreadPoolExecutor(max_workers=2)
        cases = {}           # rid -> future of its initial case
        active = []           # (req, solver, remaining)
        used = 0.0
        batch = None
        changed = False
        lat = []              # (per-step latency seconds, weight = active boxes)
        host = {"prepare": 0.0, "batch_build": 0.0, "gpu_ticks": 0.0, "retire": 0.0}
        ticks = 0
        done_points = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # arrived requests: their initial fields are built in the background
            for r in pending:
                if r.arrival > now:
                    break
                if r.rid not in cases:
                    cases[r.rid] = prep.submit(initial_case, r)
            # admission: arrived and prepared requests, while a slot and memory are free
            while pending and pending[0].arrival <= now and cases[pending[0].rid].done() \
                    and len(active) < self.max_slots and used + self._bytes(pending[0]) <= self.budget:
                r = pending.pop(0)
                tp = time.perf_counter()
                c = cases.pop(r.rid).result()
                sv = s2.Solver.from_case(c, precision=r.precision, stream=None)
                sv.set_state(c.w0)
                host["prepare"] += time.perf_counter() - tp
                active.append([r, sv, r.steps])
                used += self._bytes(r)
                r.admitted = time.perf_counter() - t0
                changed = True
            if not active:
                # idle until the next arrival or preparation
                wait = pending[0].arrival - (time.perf_counter() - t0)
                time.sleep(min(max(wait, 0.0), 0.05) if wait > 0 else 0.001)
                continue
            if changed:
                tb = time.perf_counter()
                if batch is not None:
                    batch.close()
                batch = s2.Batch([a[1] for a in active], self.stream)
                changed = False
                host["batch_build"] += time.perf_counter() - tb
            # a tick never runs past a request's end or its client's cancel
            k = min(self.k, min(self._left(a) for a in active))
            ts = time.perf_counter()
            batch.step(k)
            try:
                batch.sync()
                failed = []
            except s2.S2Error:
                # find the members whose device status is bad; the others'
                # buffers are their own, so they continue unaffected
                failed = []
                for a in active:
                    try:
                        a[1].sync()
                    except s2.S2Error as e:
                        failed.append((a, e))
            dt_tick = time.perf_counter() - ts
            host["gpu_ticks"] += dt_tick
            ticks += 1
            lat.append((dt_tick / k, len(active), k))
            for a in active:
                a[2] -= k
                done_points += a[0].points * k
            bad = {id(a) for a, _ in failed}
            retire = [(a, "failed: " + s2.s2_strerror(e.code)) for a, e in failed]
            retire += [(a, "done") for a in active if a[2] == 0 and id(a) not in bad]
            retire += [(a, "cancelled") for a in active if a[2] > 0 and id(a) not in bad
                       and a[0].cancel_after is not None and a[0].steps - a[2] >= a[0].cancel_after]
            if retire:
                tr = time.perf_counter()
                batch.close()
                batch = None
                changed = True
                for a, status in retire:
                    r, sv = a[0], a[1]
                    r.status = status
                    if self.keep and status == "done":
                        r.result = sv.get_state()
                    sv.close()
                    r.finished = time.perf_counter() - t0
                    used -= self._bytes(r)
                    active.remove(a)
                host["retire"] += time.perf_counter() - tr
            if log:
                log(ticks, len(active), len(pending), dt_tick)
        if batch is not None:
            batch.close()
        prep.shutdown()
        wall = time.perf_counter() - t0
        # per-step latency distribution, weighted by the boxes and steps of each tick
        vals = np.array([l for l, _, _ in lat])
        wts = np.array([m * k for _, m, k in lat], dtype=float)
        order = np.argsort(vals)
        cw = np.cumsum(wts[order]) / max(wts.sum(), 1.0)

        def pct(p):
            return float(vals[order][np.searchsorted(cw, p)]) if len(vals) else float("nan")

        waits = np.array([r.admitted - r.arrival for r in reqs])
        return {"requests": len(reqs), "done": sum(r.status == "done" for r in reqs),
                "cancelled": sum(r.status == "cancelled" for r in reqs),
                "failed": sum(r.status.startswith("failed") for r in reqs),
                "wall_s": wall, "point_steps": done_points,
                "throughput": done_points / wall, "ticks": ticks,
                "p50_step_latency_ms": pct(0.5) * 1e3, "p99_step_latency_ms": pct(0.99) * 1e3,
                "p50_queue_s": float(np.percentile(waits, 50)), "p99_queue_s": float(np.percentile(waits, 99)),
                "host_s": host}


def capacity(precision: str, sizes=SIZES, steps: int = 10) -> float:
    """Point-steps/s of a full batch of one box of each size (the rate the
    arrival process is tuned against)."""
    from . import s2
    reqs = [Request(rid=i, n=n, mach=0.4, re=1600.0, steps=steps, kind="tgv", precision=precision, seed=i)
            for i, n in enumerate(sizes)]
    solvers = []
    for r in reqs:
        c = initial_case(r)
        sv = s2.Solver.from_case(c, precision=precision)
        sv.set_state(c.w0)
        solvers.append(sv)
    with s2.Batch(solvers) as b:
        b.step(2)
        b.sync()
        t = time.perf_counter()
        b.step(steps)
        b.sync()
        el = time.perf_counter() - t
    for sv in solvers:
        sv.close()
    return sum(r.points for r in reqs) * steps / el


def compare(count: int = 32, seed: int = 4321, steps=(100, 1000), sizes=SIZES, stream=None) -> dict:
    """Batched serving against plain sequential FP64 solves of the same
    requests on the same GPU: the requests (all admitted at once) are
    served batched in mixed precision and batched in FP64, and solved one
    after another in FP64, each alone; reported are the three throughputs
    and the error of every mixed result against its sequential FP64 result
    (max |a - b| / max |b| per conserved field; the batched FP64 results
    equal the sequential ones exactly)."""
    from . import s2
    out = {"requests": count}
    results = {}
    for prec in ("mixed", "fp64"):
        reqs = make_requests(count, seed=seed, sizes=sizes, steps=steps, precisions=(prec,))
        r = Server(steps_per_tick=10, keep_results=True, stream=stream).run(reqs)
        out["throughput_batched_" + prec] = r["throughput"]
        results[prec] = [q.result for q in reqs]
    reqs = make_requests(count, seed=seed, sizes=sizes, steps=steps, precisions=("fp64",))
    t0 = time.perf_counter()
    seq = []
    for q in reqs:
        c = initial_case(q)
        with s2.Solver.from_case(c, precision="fp64") as sv:
            sv.set_state(c.w0)
            sv.step(q.steps)
            seq.append(sv.get_state())
    wall = time.perf_counter() - t0
    out["throughput_sequential_fp64"] = sum(q.points * q.steps for q in reqs) / wall
    out["speedup_batched_mixed_vs_sequential_fp64"] = out["throughput_batched_mixed"] / out["throughput_sequential_fp64"]
    out["speedup_batched_fp64_vs_sequential_fp64"] = out["throughput_batched_fp64"] / out["throughput_sequential_fp64"]
    # errors of the mixed results: pointwise per field (max |a-b| / max|b|),
    # and of the volume-integrated kinetic energy, per case kind; decaying
    # turbulence is chaotic, so over hundreds of steps its pointwise
    # difference grows to O(1) while the integrals stay close
    def ke(w):
        return float(np.sum(0.5 * (w[1] ** 2 + w[2] ** 2 + w[3] ** 2) / w[0]))

    for kind in ("tgv", "turb"):
        idx = [i for i, q in enumerate(reqs) if q.kind == kind]
        if not idx:
            continue
        fe = [float(np.max(np.max(np.abs(results["mixed"][i] - seq[i]), axis=(1, 2, 3)) /
                           np.max(np.abs(seq[i]), axis=(1, 2, 3)))) for i in idx]
        kd = [abs(ke(results["mixed"][i]) / ke(seq[i]) - 1.0) for i in idx]
        out["mixed_vs_fp64_" + kind] = {"cases": len(idx), "field_err_median": float(np.median(fe)),
                                        "field_err_max": float(np.max(fe)), "ke_rel_diff_max": float(np.max(kd)),
                                        "steps_median": float(np.median([reqs[i].steps for i in idx]))}
    out["batched_fp64_equals_sequential"] = all(np.array_equal(a, b) for a, b in zip(results["fp64"], seq))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--load", type=float, default=0.8, help="arrival rate as a fraction of capacity")
    ap.add_argument("--min-steps", type=int, default=100)
    ap.add_argument("--max-steps", type=int, default=1000)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--steps-per-tick", type=int, default=10)
    ap.add_argument("--compare", type=int, default=0,
                    help="instead: serve this many requests batched (mixed, FP64) and solve them sequentially in FP64")
    args = ap.parse_args(argv)
    if args.compare:
        print(json.dumps(compare(args.compare, steps=(args.min_steps, args.max_steps))))
        return
    cap = capacity(args.precision)
    reqs = make_requests(args.requests, steps=(args.min_steps, args.max_steps), precisions=(args.precision,))
    mean_work = np.mean([r.points * r.steps for r in reqs])
    rate = args.load * cap / mean_work
    poisson_arrivals(reqs, rate)
    out = Server(max_slots=args.slots, steps_per_tick=args.steps_per_tick).run(reqs)
    out.update({"precision": args.precision, "capacity": cap, "arrival_rate": rate, "load": args.load})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
