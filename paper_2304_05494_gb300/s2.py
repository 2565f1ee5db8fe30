"""Thin ctypes binding of libs2.so (include/s2.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers and back.  If the library
is missing the import fails loudly: there is no CPU fallback.

Functions keep the C names (``s2_create``, ``s2_set_state``, ``s2_step``,
``s2_get_state``, ``s2_stats``, ``s2_rhs``, ``s2_get_flags``, ``s2_sync``,
``s2_set_clock``, ``s2_destroy``, ``s2_strerror``); ``Solver`` wraps a handle.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

S2_OK, S2_EINVAL, S2_ENOMEM, S2_ECUDA, S2_ENONFINITE, S2_ETIMEOUT, S2_EBUSY = 0, -1, -2, -3, -4, -5, -6
S2_ETOOBIG, S2_EBOUNDS = -7, -8
S2_BC_PERIODIC, S2_BC_ISOTHERMAL_WALL = 0, 1
S2_HOST, S2_DEVICE = 0, 1
S2_FP64, S2_MIXED = 0, 1


class S2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, s2_strerror(code), code))


class s2_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double)]


class s2_metrics(C.Structure):
    _fields_ = [("y", C.POINTER(C.c_double))]


class s2_gas(C.Structure):
    _fields_ = [("gamma", C.c_double), ("prandtl", C.c_double), ("mach_ref", C.c_double),
                ("re_ref", C.c_double), ("visc_exp", C.c_double), ("t_ref", C.c_double),
                ("cp_coeffs", C.POINTER(C.c_double))]


class s2_bcs(C.Structure):
    _fields_ = [("x", C.c_int), ("y", C.c_int), ("z", C.c_int), ("t_wall", C.c_double),
                ("force_mass_flow", C.c_int)]


class s2_scheme(C.Structure):
    _fields_ = [("central_order", C.c_int), ("weno_order", C.c_int), ("visc_order", C.c_int),
                ("sensor_threshold", C.c_double), ("precision", C.c_int), ("cfl", C.c_double),
                ("dt_fixed", C.c_double), ("dt_every", C.c_int), ("keep", C.c_int)]


class s2_tuning(C.Structure):
    _fields_ = [("tiles", C.c_int * 3), ("flux_ctas_per_sm", C.c_int * 3), ("z_planes", C.c_int),
                ("weno_ctas_per_sm", C.c_int)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class s2_device(C.Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("ctx", C.c_void_p), ("stream", C.c_void_p),
                ("device", C.c_int)]


class s2_stats_t(C.Structure):
    _fields_ = [("t", C.c_double), ("step", C.c_longlong), ("dt", C.c_double), ("mass", C.c_double),
                ("mom", C.c_double * 3), ("energy", C.c_double), ("kinetic", C.c_double),
                ("residual_rhou", C.c_double), ("weno_frac", C.c_double), ("forcing", C.c_double),
                ("launches", C.c_longlong), ("status", C.c_int)]


S2_PROF_KINDS = 13


def _load():
    # S2_LIBRARY=checked selects the bounds-checked build (debugging, tests)
    path = _build.LIB_CHECKED if os.environ.get("S2_LIBRARY") == "checked" else _build.LIB
    if not os.path.exists(path):
        raise ImportError("%s not built; run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.s2_create.argtypes = [C.POINTER(s2_grid), C.POINTER(s2_metrics), C.POINTER(s2_gas), C.POINTER(s2_bcs),
                              C.POINTER(s2_scheme), C.POINTER(s2_device), C.POINTER(P)]
    lib.s2_create.restype = C.c_int
    lib.s2_set_state.argtypes = [P, P, C.c_int]
    lib.s2_get_state.argtypes = [P, P, C.c_int]
    lib.s2_set_primitives.argtypes = [P, P, C.c_int]
    lib.s2_get_primitives.argtypes = [P, P, C.c_int]
    lib.s2_step.argtypes = [P, C.c_int]
    lib.s2_sync.argtypes = [P]
    lib.s2_stream_states.argtypes = [P, P, C.c_longlong, P, C.c_longlong, C.c_int, C.c_int]
    lib.s2_set_clock.argtypes = [P, C.c_double, C.c_longlong, C.c_double]
    lib.s2_stats.argtypes = [P, C.POINTER(s2_stats_t)]
    lib.s2_rhs.argtypes = [P, P, C.c_int]
    lib.s2_get_flags.argtypes = [P, P, P, P]
    lib.s2_destroy.argtypes = [P]
    lib.s2_destroy.restype = None
    lib.s2_profile.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    lib.s2_profile.restype = C.c_int
    lib.s2_profile_name.argtypes = [C.c_int]
    lib.s2_profile_name.restype = C.c_char_p
    lib.s2_fma_rate.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.s2_fma_rate.restype = C.c_int
    lib.s2_cfl_dt_noalloc.argtypes = [C.POINTER(s2_grid), C.POINTER(s2_gas), P, P, C.c_double, P, P]
    lib.s2_cfl_dt_noalloc.restype = C.c_int
    lib.s2_batch_create_ex.argtypes = [C.POINTER(P), C.c_int, P, C.c_int, C.POINTER(P)]
    lib.s2_batch_create_ex.restype = C.c_int
    lib.s2_batch_launches.argtypes = [P]
    lib.s2_batch_launches.restype = C.c_longlong
    lib.s2_batch_create.argtypes = [C.POINTER(P), C.c_int, P, C.POINTER(P)]
    lib.s2_batch_create.restype = C.c_int
    lib.s2_batch_step.argtypes = [P, C.c_int]
    lib.s2_batch_step.restype = C.c_int
    lib.s2_batch_sync.argtypes = [P]
    lib.s2_batch_sync.restype = C.c_int
    lib.s2_batch_destroy.argtypes = [P]
    lib.s2_batch_destroy.restype = None
    lib.s2_set_tiles.argtypes = [P, C.POINTER(C.c_int)]
    lib.s2_set_tiles.restype = C.c_int
    lib.s2_set_tuning.argtypes = [P, C.POINTER(s2_tuning)]
    lib.s2_set_tuning.restype = C.c_int
    lib.s2_get_tuning.argtypes = [P, C.POINTER(s2_tuning)]
    lib.s2_get_tuning.restype = C.c_int
    lib.s2_strerror.argtypes = [C.c_int]
    lib.s2_strerror.restype = C.c_char_p
    for f in ("s2_set_state", "s2_get_state", "s2_step", "s2_sync", "s2_set_clock", "s2_stats", "s2_rhs",
              "s2_get_flags", "s2_stream_states"):
        getattr(lib, f).restype = C.c_int
    del dp
    return lib


_lib = _load()
LIB_PATH = _build.LIB


def _check(code: int, what: str) -> int:
    if code != S2_OK:
        raise S2Error(code, what)
    return code


def s2_strerror(code: int) -> str:
    return _lib.s2_strerror(code).decode()


def s2_create(grid, metrics, gas, bcs, scheme, dev=None):
    h = C.c_void_p()
    rc = _lib.s2_create(C.byref(grid), C.byref(metrics) if metrics is not None else None, C.byref(gas),
                        C.byref(bcs), C.byref(scheme), C.byref(dev) if dev is not None else None, C.byref(h))
    _check(rc, "s2_create")
    return h


def _ptr(a) -> tuple:
    """(pointer, where, keepalive) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("need a C-contiguous float64 array")
        return a.ctypes.data, S2_HOST, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("need a contiguous float64 tensor")
        return a.data_ptr(), (S2_DEVICE if a.is_cuda else S2_HOST), a
    raise TypeError("unsupported buffer type %r" % type(a))


def s2_set_state(h, w) -> None:
    p, where, _ = _ptr(w)
    _check(_lib.s2_set_state(h, p, where), "s2_set_state")


def s2_get_state(h, out) -> None:
    p, where, _ = _ptr(out)
    _check(_lib.s2_get_state(h, p, where), "s2_get_state")


def s2_stream_states(h, w_in, in_stride: int, w_out, out_stride: int, count: int, nsteps: int) -> None:
    pi, _, _ = _ptr(w_in)
    po, _, _ = _ptr(w_out)
    _check(_lib.s2_stream_states(h, pi, in_stride, po, out_stride, count, nsteps), "s2_stream_states")


def s2_set_primitives(h, prim) -> None:
    p, where, _ = _ptr(prim)
    _check(_lib.s2_set_primitives(h, p, where), "s2_set_primitives")


def s2_get_primitives(h, out) -> None:
    p, where, _ = _ptr(out)
    _check(_lib.s2_get_primitives(h, p, where), "s2_get_primitives")


def s2_step(h, n: int) -> None:
    _check(_lib.s2_step(h, int(n)), "s2_step")


def s2_sync(h) -> None:
    _check(_lib.s2_sync(h), "s2_sync")


def s2_set_clock(h, t: float, step: int, dt: float) -> None:
    _check(_lib.s2_set_clock(h, t, step, dt), "s2_set_clock")


def s2_set_tiles(h, tiles) -> None:
    arr = (C.c_int * 3)(*[int(t) for t in tiles])
    _check(_lib.s2_set_tiles(h, arr), "s2_set_tiles")


def s2_set_tuning(h, tiles=(0, 0, 0), flux_ctas_per_sm=0, z_planes=0, weno_ctas_per_sm=0) -> None:
    """flux_ctas_per_sm: one value for the three directions or one per direction."""
    cps = [flux_ctas_per_sm] * 3 if np.isscalar(flux_ctas_per_sm) else list(flux_ctas_per_sm)
    t = s2_tuning((C.c_int * 3)(*[int(x) for x in tiles]), (C.c_int * 3)(*[int(x) for x in cps]), int(z_planes),
                  int(weno_ctas_per_sm))
    _check(_lib.s2_set_tuning(h, C.byref(t)), "s2_set_tuning")


def s2_get_tuning(h) -> dict:
    t = s2_tuning()
    _check(_lib.s2_get_tuning(h, C.byref(t)), "s2_get_tuning")
    return {"tiles": list(t.tiles), "flux_ctas_per_sm": list(t.flux_ctas_per_sm), "z_planes": t.z_planes,
            "weno_ctas_per_sm": t.weno_ctas_per_sm}


def s2_stats(h) -> dict:
    st = s2_stats_t()
    rc = _lib.s2_stats(h, C.byref(st))
    out = {"t": st.t, "step": st.step, "dt": st.dt, "mass": st.mass, "mom": list(st.mom),
           "energy": st.energy, "kinetic": st.kinetic, "residual_rhou": st.residual_rhou,
           "weno_frac": st.weno_frac, "forcing": st.forcing, "launches": st.launches, "status": st.status}
    if rc not in (S2_OK, S2_ENONFINITE):
        _check(rc, "s2_stats")
    return out


def s2_rhs(h, out) -> None:
    p, where, _ = _ptr(out)
    _check(_lib.s2_rhs(h, p, where), "s2_rhs")


def s2_get_flags(h, fx: Optional[np.ndarray], fy: Optional[np.ndarray], fz: Optional[np.ndarray]) -> None:
    ps = [a.ctypes.data if a is not None else None for a in (fx, fy, fz)]
    _check(_lib.s2_get_flags(h, *ps), "s2_get_flags")


def s2_profile_name(kind: int) -> str:
    r = _lib.s2_profile_name(kind)
    return r.decode() if r else ""


def s2_profile(h, n: int) -> dict:
    """n steps with per-kernel-class CUDA event timing: {name: (ms, launches)}."""
    ms = (C.c_double * S2_PROF_KINDS)()
    cnt = (C.c_longlong * S2_PROF_KINDS)()
    _check(_lib.s2_profile(h, int(n), ms, cnt), "s2_profile")
    return {s2_profile_name(k): (ms[k], cnt[k]) for k in range(S2_PROF_KINDS)}


def s2_fma_rate(precision: str = "fp64", device: int = -1) -> float:
    """Issue-limited FMA rate of the GPU in GFLOP/s (double or single precision)."""
    g = C.c_double(0.0)
    _check(_lib.s2_fma_rate(S2_FP64 if precision == "fp64" else S2_MIXED, int(device), C.byref(g)), "s2_fma_rate")
    return g.value


def s2_cfl_dt_noalloc(grid, gas, w, eta_y, cfl: float, dt, stream=None) -> int:
    """Allocation-free CFL dt; w, eta_y (or None) and dt are CUDA tensors.
    Returns the status code (no exception, so callers can test it)."""
    return _lib.s2_cfl_dt_noalloc(C.byref(grid), C.byref(gas), w.data_ptr(),
                                  eta_y.data_ptr() if eta_y is not None else None, cfl, dt.data_ptr(), stream)


S2_BATCH_WORKLIST, S2_BATCH_BRANCHES, S2_BATCH_WORKLIST_ALL = 0, 1, 2
_BATCH_MODES = {"worklist": S2_BATCH_WORKLIST, "branches": S2_BATCH_BRANCHES, "worklist_all": S2_BATCH_WORKLIST_ALL}


def s2_batch_create(handles, stream=None, mode: str = "worklist"):
    """mode: "worklist" (one launch per kernel for all boxes of a group;
    members of 64^3 points or more keep their own launches), "worklist_all"
    (every member in the work list) or "branches" (each member's own
    launches as concurrent graph branches)."""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    m = _BATCH_MODES[mode]
    _check(_lib.s2_batch_create_ex(arr, len(handles), stream, m, C.byref(b)), "s2_batch_create")
    return b


def s2_batch_create_ex(handles, stream=None, mode: int = S2_BATCH_WORKLIST):
    """The C call with its integer mode (S2_BATCH_WORKLIST, S2_BATCH_BRANCHES
    or S2_BATCH_WORKLIST_ALL)."""
    name = {v: k for k, v in _BATCH_MODES.items()}[int(mode)]
    return s2_batch_create(handles, stream, name)


def s2_batch_launches(b) -> int:
    return int(_lib.s2_batch_launches(b))


def s2_batch_step(b, n: int) -> None:
    _check(_lib.s2_batch_step(b, int(n)), "s2_batch_step")


def s2_batch_sync(b) -> None:
    _check(_lib.s2_batch_sync(b), "s2_batch_sync")


def s2_batch_destroy(b) -> None:
    _lib.s2_batch_destroy(b)


class Batch:
    """Owning wrapper of a batch of solvers (destroyed before its members)."""

    def __init__(self, solvers, stream=None, mode: str = "worklist"):
        self.solvers = list(solvers)
        self.b = s2_batch_create([sv.h for sv in self.solvers], stream, mode)

    @property
    def launches_per_step(self) -> int:
        return s2_batch_launches(self.b)

    def step(self, n: int = 1):
        s2_batch_step(self.b, n)

    def sync(self):
        s2_batch_sync(self.b)

    def close(self):
        if self.b:
            s2_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def s2_destroy(h) -> None:
    _lib.s2_destroy(h)


class Solver:
    """Owning wrapper of one solver handle."""

    def __init__(self, nx, ny, nz, lx, ly, lz, *, y=None, gamma=1.4, prandtl=0.72, mach=0.1, re=1600.0,
                 visc_exp=0.76, t_ref=1.0, wall_y=False, t_wall=1.0, force=False, weno_order=0,
                 threshold=0.2, cfl=0.8, dt_fixed=0.0, dt_every=10, stream=None, device=-1, precision="fp64",
                 central_order=6, visc_order=6, cp_coeffs=None, keep=0):
        self.shape = (5, nz, ny, nx)
        self.n = nx * ny * nz
        self.precision = precision
        grid = s2_grid(nx, ny, nz, lx, ly, lz)
        self._y = None
        met = s2_metrics()
        if y is not None:
            self._y = np.ascontiguousarray(y, dtype=np.float64)
            met.y = self._y.ctypes.data_as(C.POINTER(C.c_double))
        gas = s2_gas(gamma, prandtl, mach, re, visc_exp, t_ref)
        if cp_coeffs is not None:
            # thermally perfect gas: a_{-2..4} of c_p/R = sum_l a_l T^l (read during s2_create)
            cpc = np.ascontiguousarray(cp_coeffs, dtype=np.float64)
            if cpc.shape != (7,):
                raise ValueError("cp_coeffs needs the 7 coefficients a_-2 .. a_4")
            gas.cp_coeffs = cpc.ctypes.data_as(C.POINTER(C.c_double))
        bcs = s2_bcs(S2_BC_PERIODIC, S2_BC_ISOTHERMAL_WALL if wall_y else S2_BC_PERIODIC, S2_BC_PERIODIC,
                     t_wall, 1 if force else 0)
        prec = {"fp64": S2_FP64, "mixed": S2_MIXED}[precision]
        sch = s2_scheme(central_order, weno_order, visc_order, threshold, prec, cfl, dt_fixed, dt_every, keep)
        dev = s2_device()
        dev.stream = stream
        dev.device = device
        self.h = s2_create(grid, met, gas, bcs, sch, dev)

    @classmethod
    def from_case(cls, case, **kw):
        args = dict(y=case.y, gamma=case.gamma, prandtl=case.prandtl, mach=case.mach, re=case.re,
                    visc_exp=case.visc_exp, t_ref=case.t_ref, wall_y=case.wall_y, t_wall=case.t_wall,
                    force=case.force, weno_order=case.weno_order, threshold=case.threshold, cfl=case.cfl,
                    dt_fixed=case.dt_fixed, dt_every=case.dt_every,
                    central_order=getattr(case, "central_order", 6), visc_order=getattr(case, "visc_order", 6))
        args.update(kw)
        return cls(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, **args)

    def _fits(self, a):
        """The library reads or writes 5 nx ny nz doubles: refuse other sizes."""
        shape = tuple(a.shape)
        if shape != self.shape and shape != (5 * self.n,):
            raise ValueError("state buffer of shape %s, need %s" % (shape, self.shape))
        return a

    def set_state(self, w):
        s2_set_state(self.h, self._fits(w))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        s2_get_state(self.h, self._fits(out))
        return out

    def stream_states(self, w_in, w_out, nsteps: int, count: Optional[int] = None):
        """Copy in, advance nsteps and copy out count states, the copies
        overlapping the steps (s2_stream_states).  w_in / w_out: a stack of
        states (count, 5, nz, ny, nx), or one state (5, nz, ny, nx) used for
        every j (count then required; w_out then holds the last result)."""
        strides = []
        for a in (w_in, w_out):
            shape = tuple(a.shape)
            if shape == self.shape:
                if count is None:
                    raise ValueError("count is needed when a buffer holds one state")
                strides.append(0)
            elif len(shape) == 5 and shape[1:] == self.shape:
                if count is None:
                    count = shape[0]
                if shape[0] < count:
                    raise ValueError("buffer of %d states for count %d" % (shape[0], count))
                strides.append(5 * self.n)
            else:
                raise ValueError("state stack of shape %s, need (count,) + %s" % (shape, self.shape))
        s2_stream_states(self.h, w_in, strides[0], w_out, strides[1], count, nsteps)
        return w_out

    def set_primitives(self, prim):
        """State from primitive fields (rho, u, v, w, T), shape (5, nz, ny, nx)."""
        s2_set_primitives(self.h, self._fits(prim))

    def get_primitives(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        s2_get_primitives(self.h, self._fits(out))
        return out

    def step(self, n: int = 1):
        s2_step(self.h, n)

    def sync(self):
        s2_sync(self.h)

    def set_tiles(self, tiles):
        s2_set_tiles(self.h, tiles)

    def set_tuning(self, **knobs):
        """tiles, flux_ctas_per_sm, z_planes, weno_ctas_per_sm (see s2_tuning)."""
        cur = s2_get_tuning(self.h)
        cur.update(knobs)
        s2_set_tuning(self.h, **cur)

    def get_tuning(self) -> dict:
        return s2_get_tuning(self.h)

    def set_clock(self, t, step, dt):
        s2_set_clock(self.h, t, step, dt)

    def stats(self) -> dict:
        return s2_stats(self.h)

    def rhs(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        s2_rhs(self.h, self._fits(out))
        return out

    def flags(self):
        nz, ny, nx = self.shape[1:]
        fx = np.zeros((nz, ny, nx + 1), np.uint8)
        fy = np.zeros((nz, ny + 1, nx), np.uint8)
        fz = np.zeros((nz + 1, ny, nx), np.uint8)
        s2_get_flags(self.h, fx, fy, fz)
        return fx, fy, fz

    def profile(self, n: int) -> dict:
        return s2_profile(self.h, n)

    def close(self):
        if self.h:
            s2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
