"""Operation tally of the CPU oracle: floating-point operations per grid
point of each part of the method, as the oracle's direct formulation
performs them.  TEST INFRASTRUCTURE ONLY (used by tests/ to check the
algorithmic operation counts that the benchmark's roofline quotes).

The counting build compiles ``s2_oracle.c`` unchanged as C++ with every
double replaced by the counting type of ``count_double.hpp`` (same layout,
bit-identical results); the oracle's section markers attribute each
operation to a part of the method.  Adds and subtracts, multiplies,
divides, square roots and transcendental calls (pow, log, exp) are counted
separately; the flop count is their sum (each counted as one).  Maxima,
absolute values and comparisons are not counted.

    python -m oracle.tally          # prints the table for the benchmark channel's scheme
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "s2_oracle_tally.cpp")
LIB = os.path.join(O.BUILD_DIR, "liboracle_tally.so")
SECTIONS = ["prims", "sensor", "central", "weno", "visc_grad", "visc", "force", "update", "dt", "prims_hc", "ghost"]
KINDS = ["add", "mul", "div", "sqrt", "trans"]


def build(force: bool = False) -> str:
    deps = [SRC, O.SRC, os.path.join(HERE, "count_double.hpp")]
    os.makedirs(O.BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(d) for d in deps):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                        "-Wno-return-type-c-linkage", SRC, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = O.load(build())
        _lib.or_tally_reset.argtypes = []
    return _lib


def _counts():
    arr = (C.c_longlong * (16 * 5)).in_dll(lib(), "or_tally")
    a = np.array(arr[:], dtype=np.int64).reshape(16, 5)
    return {sec: dict(zip(KINDS, a[i].tolist())) for i, sec in enumerate(SECTIONS)}


def run(fn):
    """Counts of the operations performed by fn() (which calls the oracle
    through oracle.oracle while the counting library is loaded)."""
    old = O._lib
    O._lib = lib()
    try:
        lib().or_tally_reset()
        out = fn()
    finally:
        O._lib = old
    return _counts(), out


def flops(c: dict) -> int:
    return int(sum(c.values()))


def per_point_step(problem: O.Problem, w: np.ndarray, weno_frac: float):
    """Algorithmic flops per grid point of one RK3 step (three RHS
    evaluations and updates) of problem's scheme, per part of the method,
    for a hybrid scheme with the given fraction of WENO interfaces
    (flagged interfaces / 3N).  Central-only and WENO-everywhere RHS
    evaluations of w give the cost of a central and of a WENO interface;
    the hybrid mixes them.  Also returns the per-interface figures."""
    n = problem.nx * problem.ny * problem.nz
    pc = O.Problem(**{**problem.__dict__, "threshold": 1e30, "_y_buf": None, "_cp_buf": None})
    pw = O.Problem(**{**problem.__dict__, "threshold": -1.0, "_y_buf": None, "_cp_buf": None})
    cc, _ = run(lambda: O.rhs(pc, w))
    cw, _ = run(lambda: O.rhs(pw, w))
    cs, _ = run(lambda: O.step(pc, w, 1, dt_fixed=1e-6))
    cdt, _ = run(lambda: O.dt(pc, w, 0.8))
    # H and c are formed on interior and face-ghost points; edges and corners
    # of the padded arrays hold T = 0, where only H is formed (8 operations
    # for a calorically perfect gas, 6 for a thermally perfect one)
    gh = 4
    nx, ny, nz = problem.nx, problem.ny, problem.nz
    faces = 2 * gh * (ny * nz + nx * nz + nx * ny)
    edges = (nx + 2 * gh) * (ny + 2 * gh) * (nz + 2 * gh) - n - faces
    hc = (flops(cc["prims_hc"]) - (8 if problem.cp_coef is None else 6) * edges) / (n + faces)
    interfaces = ((problem.nx + 1) * problem.ny * problem.nz + problem.nx * (problem.ny + 1) * problem.nz
                  + problem.nx * problem.ny * (problem.nz + 1))
    central_if = (flops(cc["central"]) - flops(cw["central"])) / interfaces  # one central interface flux
    weno_if = flops(cw["weno"]) / interfaces                                 # one WENO interface flux
    diff_pp = flops(cw["central"]) / n                                       # flux differences per point
    frac_if = weno_frac * 3 * n / interfaces
    stage = {
        "prims": flops(cc["prims"]) / n + hc,
        "grad": flops(cc["sensor"]) / n,
        "flux": diff_pp + interfaces / n * ((1 - frac_if) * central_if + frac_if * weno_if),
        "visc": flops(cc["visc"]) / n,
        "visc_grad": flops(cc["visc_grad"]) / n,
        "force": flops(cc["force"]) / n,
        "update": flops(cs["update"]) / (3 * n),
    }
    step = {k: 3 * v for k, v in stage.items()}
    step["dt"] = flops(cdt["dt"]) / n
    return {"per_point_stage": stage, "h_and_c_per_point": hc, "per_point_step": step, "central_interface": central_if,
            "weno_interface": weno_if, "flux_difference_per_point": diff_pp, "weno_frac": weno_frac}


if __name__ == "__main__":
    import json
    import sys

    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2304_05494_gb300 import workloads as W

    case = W.channel(32, 24, 16, seed=4)
    pr = O.Problem(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, y=case.y, mach=case.mach, re=case.re,
                   visc_exp=case.visc_exp, prandtl=case.prandtl, wall_y=case.wall_y, t_wall=case.t_wall,
                   force=case.force, weno_order=case.weno_order, threshold=case.threshold)
    frac = float(sys.argv[1]) if len(sys.argv) > 1 else 0.013
    print(json.dumps(per_point_step(pr, case.w0, frac), indent=1))
