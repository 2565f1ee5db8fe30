"""Tile-shape autotuner for the flux kernels.

The paper tunes the CUDA block shape of its kernels by hand (launch bounds
128x1..640, block 128x3 chosen, Sec. 4.1, Table 3).  Here each flux
direction has two tile shapes compiled in (see s2_set_tiles); the tuner
times both on the caller's problem with the library's own CUDA-event trace
(s2_profile), keeps the faster per direction, and caches the choice in a
JSON file keyed by grid, precision, WENO order and GPU name.

Tuning advances the solver; tune_solver() restores the given state and
clock afterwards, so it can run right before a production run.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Optional, Sequence

import numpy as np

CACHE_PATH = os.environ.get("S2_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))
_lock = threading.Lock()
_DIRS = ("flux_x", "flux_y", "flux_z")


def gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:  # pragma: no cover - informational only
        return "unknown"


def key(shape: Sequence[int], precision: str, weno: int, gpu: Optional[str] = None) -> str:
    nx, ny, nz = shape
    return "%dx%dx%d|%s|weno%d|%s" % (nx, ny, nz, precision, weno, gpu or gpu_name())


def load_cache(path: str = CACHE_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE_PATH) -> None:
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(times: dict) -> list:
    """Per direction the variant with the smaller time; times[v][dir] = ms."""
    out = []
    for d in _DIRS:
        best = min(times, key=lambda v: times[v][d])
        out.append(int(best))
    return out


def tune_solver(sv, w: np.ndarray, steps: int = 3, variants=(0, 1)) -> tuple:
    """Time every tile variant on solver sv from state w; set the fastest
    per direction; restore w and the clock.  Returns (tiles, times)."""
    times = {}
    for v in variants:
        sv.set_tiles([v, v, v])
        sv.set_state(w)
        sv.set_clock(0.0, 0, 0.0)
        sv.profile(1)  # warm-up
        prof = sv.profile(steps)
        times[v] = {d: prof[d][0] / max(prof[d][1], 1) for d in _DIRS}
    tiles = choose(times)
    sv.set_tiles(tiles)
    sv.set_state(w)
    sv.set_clock(0.0, 0, 0.0)
    return tiles, times


def tiles_for(sv, w: np.ndarray, shape, precision: str, weno: int, path: str = CACHE_PATH, steps: int = 3) -> list:
    """Cached tile choice for this problem class, tuning on a miss."""
    k = key(shape, precision, weno)
    with _lock:
        cache = load_cache(path)
        if k in cache:
            tiles = cache[k]["tiles"]
            sv.set_tiles(tiles)
            return tiles
    tiles, times = tune_solver(sv, w, steps)
    with _lock:
        cache = load_cache(path)
        cache[k] = {"tiles": tiles, "ms_per_launch": {str(v): t for v, t in times.items()}}
        save_cache(cache, path)
    return tiles
