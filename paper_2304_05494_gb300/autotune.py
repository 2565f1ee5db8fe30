"""Launch-shape autotuner.

The paper tunes the CUDA block shape of its kernels by hand (launch bounds
128x1..640, block 128x3 chosen, Sec. 4.1, Table 3) and its translator takes
the launch configuration from a configuration file (Sec. 3.3).  Here the
knobs of s2_tuning are searched on the caller's problem, timed with the
library's own CUDA-event trace (s2_profile) per kernel class:

* the flux tile shape of each direction (two compiled per direction: the
  tile length along the direction against the pencils across), timed per
  direction (flux_x, flux_y, flux_z);
* single precision: the resident CTAs per multiprocessor of the persistent
  flux grid of each direction (1..4, or all that fit), each direction
  timed on its own flux class;
* single precision: the z-planes each CTA of the z-marching gradient and
  viscous passes walks (4, 8, 12, 16, 24), timed on grad + visc;
* the CTAs per multiprocessor of the WENO kernels' grids (4..32), timed on
  the WENO class (hybrid schemes only).

Each knob is chosen by itself with the others at their current value
(coordinate descent: the knobs act on different kernels), and the choice
is cached in a JSON file keyed by grid, precision, WENO order and GPU name.
Results do not depend on the knobs (tested bit for bit).  Tuning advances
the solver; tune_solver() restores the given state and clock afterwards, so
it can run right before a production run.
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
FLUX_CTAS = (1, 2, 3, 4, 0)
Z_PLANES = (4, 8, 12, 16, 24)
WENO_CTAS = (4, 8, 16, 32)


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


def _profile(sv, w, steps) -> dict:
    """Per-class (ms, launches) of `steps` steps from state w."""
    sv.set_state(w)
    sv.set_clock(0.0, 0, 0.0)
    sv.profile(1)  # warm-up (and graph rebuild)
    return sv.profile(steps)


def _time(sv, w, steps, classes) -> float:
    """ms per step of the given kernel classes from state w."""
    prof = _profile(sv, w, steps)
    return sum(prof[c][0] for c in classes if c in prof) / steps


def tune_solver(sv, w: np.ndarray, steps: int = 3, variants=(0, 1), mixed: Optional[bool] = None,
                weno: Optional[bool] = None) -> tuple:
    """Search the launch knobs on solver sv from state w; set the best;
    restore w and the clock.  Returns (tuning, times)."""
    times = {"tiles": {}}
    for v in variants:
        sv.set_tuning(tiles=[v, v, v])
        sv.set_state(w)
        sv.set_clock(0.0, 0, 0.0)
        sv.profile(1)
        prof = sv.profile(steps)
        times["tiles"][v] = {d: prof[d][0] / max(prof[d][1], 1) for d in _DIRS}
    sv.set_tuning(tiles=choose(times["tiles"]))
    if mixed is None:
        mixed = getattr(sv, "precision", "fp64") == "mixed"
    searches = []
    if mixed:
        # one pass over the values sets the three directions alike; each
        # direction's grid only changes its own kernel, so each takes the
        # value that timed best for its own class
        t = {}
        for v in FLUX_CTAS:
            sv.set_tuning(flux_ctas_per_sm=v)
            prof = _profile(sv, w, steps)
            t[v] = {d: prof[d][0] / steps for d in _DIRS if d in prof}
        sv.set_tuning(flux_ctas_per_sm=[min(t, key=lambda v: t[v][d]) for d in _DIRS])
        times["flux_ctas_per_sm"] = t
        searches.append(("z_planes", Z_PLANES, ("grad", "visc")))
    if weno:
        searches.append(("weno_ctas_per_sm", WENO_CTAS, ("weno",)))
    for knob, values, classes in searches:
        t = {}
        for v in values:
            sv.set_tuning(**{knob: v})
            t[v] = _time(sv, w, steps, classes)
        best = min(t, key=t.get)
        sv.set_tuning(**{knob: best})
        times[knob] = t
    sv.set_state(w)
    sv.set_clock(0.0, 0, 0.0)
    return sv.get_tuning(), times


def tuning_for(sv, w: np.ndarray, shape, precision: str, weno: int, path: str = CACHE_PATH, steps: int = 3) -> dict:
    """Cached launch knobs for this problem class, tuning on a miss."""
    k = key(shape, precision, weno)
    with _lock:
        cache = load_cache(path)
        if k in cache and "tuning" in cache[k]:
            t = cache[k]["tuning"]
            sv.set_tuning(**t)
            return t
    t, times = tune_solver(sv, w, steps, mixed=precision == "mixed", weno=weno > 0)
    with _lock:
        cache = load_cache(path)
        cache[k] = {"tuning": t, "tiles": t["tiles"],
                    "ms": {kn: {str(v): tv for v, tv in val.items()} for kn, val in times.items()}}
        save_cache(cache, path)
    return t


def tiles_for(sv, w: np.ndarray, shape, precision: str, weno: int, path: str = CACHE_PATH, steps: int = 3) -> list:
    """Cached tile choice (the tile knob of tuning_for)."""
    return tuning_for(sv, w, shape, precision, weno, path, steps)["tiles"]
