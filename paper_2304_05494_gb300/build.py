"""Build libs2.so (the CUDA solver behind include/s2.h) for sm_103a, in tree.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  No CMake.

The checked variant libs2_checked.so (-DS2_CHECKED) tests the index
arithmetic of every kernel against its array before each access and
reports S2_EBOUNDS instead of touching memory out of range; the binding
loads it when S2_LIBRARY=checked.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libs2.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libs2_checked.so")
SOURCES = ["s2_solver.cu", "s2_flux.cu", "s2_visc.cu", "s2_noalloc.cu", "s2_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    files.append(os.path.join(ROOT, "include", "s2.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _build_one(lib: str, defines: list, verbose: bool) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tag = os.path.splitext(os.path.basename(lib))[0]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, "%s_%s.o" % (tag, os.path.splitext(src)[0]))
        cmd = [nvcc, *ARCH, *FLAGS, *defines, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Build libs2.so and (checked=True) libs2_checked.so, each when out of
    date; returns the path of libs2.so."""
    jobs = []
    if force or not up_to_date(LIB):
        jobs.append((LIB, []))
    if checked and (force or not up_to_date(LIB_CHECKED)):
        jobs.append((LIB_CHECKED, ["-DS2_CHECKED"]))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _build_one(j[0], j[1], verbose), jobs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
