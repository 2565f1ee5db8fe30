"""ctypes binding of the plain FP64 CPU oracle (``oracle/s2_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

The oracle follows paper Sec. 2 ("Numerical Methods"): split-form central
convective flux, Ducros-type sensor, characteristic WENO with Lax-Friedrichs
splitting, Laplacian-form viscous terms, low-storage RK3; plus the forcing and
dt reductions of Table 2.  States are numpy float64 arrays of shape
(5, nz, ny, nx): (rho, rho u, rho v, rho w, rho E).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "s2_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

CONV, VISC, FORCE = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, OpenMP over k, no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("y", C.POINTER(C.c_double)),
        ("gamma", C.c_double), ("prandtl", C.c_double), ("mach", C.c_double),
        ("re", C.c_double), ("visc_exp", C.c_double), ("t_ref", C.c_double),
        ("bc_y", C.c_int), ("t_wall", C.c_double),
        ("force", C.c_int), ("weno_order", C.c_int), ("threshold", C.c_double),
        ("central_order", C.c_int), ("visc_order", C.c_int),
        ("cp_coef", C.POINTER(C.c_double)),
        ("keep", C.c_int),
    ]


_lib = None


def load(path: str) -> C.CDLL:
    """Load an oracle library built from ``s2_oracle.c`` and declare its entry
    points (the tests also load deliberately broken copies this way)."""
    lb = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    bp = C.POINTER(C.c_ubyte)
    lb.or_rhs.argtypes = [C.POINTER(_Cfg), dp, dp, bp, bp, bp, C.c_int, dp]
    lb.or_rhs.restype = C.c_int
    lb.or_rhs_given_flags.argtypes = [C.POINTER(_Cfg), dp, dp, bp, bp, bp, C.c_int]
    lb.or_rhs_given_flags.restype = C.c_int
    lb.or_sensor.argtypes = [C.POINTER(_Cfg), dp, dp, dp]
    lb.or_sensor.restype = C.c_int
    lb.or_dt.argtypes = [C.POINTER(_Cfg), dp, C.c_double]
    lb.or_dt.restype = C.c_double
    lb.or_step.argtypes = [C.POINTER(_Cfg), dp, C.c_int, C.c_double, C.c_double, C.c_int,
                           C.POINTER(C.c_longlong), dp]
    lb.or_step.restype = C.c_int
    lb.or_metric.argtypes = [C.POINTER(_Cfg), dp, dp]
    lb.or_weno_rec.argtypes = [C.c_int, dp]
    lb.or_weno_rec.restype = C.c_double
    lb.or_weno_parts.argtypes = [C.c_int, dp, dp, dp]
    lb.or_weno_parts.restype = C.c_int
    lb.or_eigvec.argtypes = [C.c_double, C.c_int, dp, C.c_double, dp, dp]
    lb.or_eigvec.restype = C.c_double
    lb.or_eigvec_tp.argtypes = [C.c_double, C.c_double, C.c_int, dp, C.c_double, dp, dp]
    lb.or_eigvec_tp.restype = C.c_double
    lb.or_thermo.argtypes = [C.POINTER(_Cfg), C.c_double, dp, dp, dp]
    lb.or_thermo.restype = C.c_int
    lb.or_temperature.argtypes = [C.POINTER(_Cfg), C.c_double, C.c_int, C.c_double]
    lb.or_temperature.restype = C.c_double
    lb.or_roe_state.argtypes = [C.POINTER(_Cfg), dp, dp, dp]
    lb.or_roe_state.restype = C.c_int
    lb.or_rk3_scalar.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
    lb.or_rk3_scalar.restype = C.c_double
    return lb


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _bp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_ubyte))


@dataclass
class Problem:
    """One solver configuration (grid, gas, boundaries, scheme)."""
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    y: Optional[np.ndarray] = None       # ny node ordinates, None = uniform
    gamma: float = 1.4
    prandtl: float = 0.72
    mach: float = 0.1
    re: float = 1600.0                   # <= 0: inviscid
    visc_exp: float = 0.76
    t_ref: float = 1.0
    wall_y: bool = False                 # isothermal no-slip walls at y = -ly/2, +ly/2
    t_wall: float = 1.0
    force: bool = False
    weno_order: int = 0                  # 0, 1, 3, 5, 7
    threshold: float = 0.2
    central_order: int = 6               # 2, 4, 6, 8
    visc_order: int = 6                  # 2, 4, 6, 8
    # thermally perfect gas: a_{-2..4} of c_p/R = sum_l a_l T^l; None = calorically perfect
    cp_coef: Optional[np.ndarray] = None
    # central flux: 0 split form; n >= 1 KEEP-n (log means from n series terms); -1 KEEP, exact log means
    keep: int = 0
    _y_buf: Optional[np.ndarray] = field(default=None, repr=False)
    _cp_buf: Optional[np.ndarray] = field(default=None, repr=False)

    def cfg(self) -> _Cfg:
        if self.wall_y and self.ny < 4:
            raise ValueError("walls need ny >= 4")
        c = _Cfg()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.lx, c.ly, c.lz = self.lx, self.ly, self.lz
        if self.y is not None:
            self._y_buf = np.ascontiguousarray(self.y, dtype=np.float64)
            assert self._y_buf.shape == (self.ny,)
            c.y = _dp(self._y_buf)
        else:
            c.y = None
        c.gamma, c.prandtl, c.mach = self.gamma, self.prandtl, self.mach
        c.re, c.visc_exp, c.t_ref = self.re, self.visc_exp, self.t_ref
        c.bc_y = 1 if self.wall_y else 0
        c.t_wall = self.t_wall
        c.force = 1 if self.force else 0
        c.weno_order = self.weno_order
        c.threshold = self.threshold
        c.central_order = self.central_order
        c.visc_order = self.visc_order
        if self.cp_coef is not None:
            self._cp_buf = np.ascontiguousarray(self.cp_coef, dtype=np.float64)
            assert self._cp_buf.shape == (7,)
            c.cp_coef = _dp(self._cp_buf)
        else:
            c.cp_coef = None
        c.keep = self.keep
        return c

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)


def _state(p: Problem, w: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != p.shape:
        raise ValueError("state shape %s != %s" % (w.shape, p.shape))
    return w


def rhs(p: Problem, w: np.ndarray, terms: int = CONV | VISC | FORCE, flags: bool = False):
    """R(w).  With flags=True also returns the per-direction interface WENO
    flags, shapes (nz, ny, nx+1), (nz, ny+1, nx), (nz+1, ny, nx)."""
    w = _state(p, w)
    out = np.zeros_like(w)
    cfg = p.cfg()
    fx = fy = fz = None
    if flags:
        fx = np.zeros((p.nz, p.ny, p.nx + 1), np.uint8)
        fy = np.zeros((p.nz, p.ny + 1, p.nx), np.uint8)
        fz = np.zeros((p.nz + 1, p.ny, p.nx), np.uint8)
    fo = C.c_double(0.0)
    rc = lib().or_rhs(C.byref(cfg), _dp(w), _dp(out), _bp(fx), _bp(fy), _bp(fz), terms, C.byref(fo))
    if rc:
        raise MemoryError("oracle rhs failed")
    if flags:
        return out, (fx, fy, fz)
    return out


def rhs_given_flags(p: Problem, w: np.ndarray, flags, terms: int = CONV | VISC | FORCE):
    """R(w) with the interface flags (fx, fy, fz) imposed instead of decided
    by the sensor (same layout as rhs(..., flags=True) returns)."""
    w = _state(p, w)
    out = np.zeros_like(w)
    cfg = p.cfg()
    fx, fy, fz = [np.ascontiguousarray(f, dtype=np.uint8) for f in flags]
    assert fx.shape == (p.nz, p.ny, p.nx + 1) and fy.shape == (p.nz, p.ny + 1, p.nx)
    assert fz.shape == (p.nz + 1, p.ny, p.nx)
    if lib().or_rhs_given_flags(C.byref(cfg), _dp(w), _dp(out), _bp(fx), _bp(fy), _bp(fz), terms):
        raise MemoryError("oracle rhs failed")
    return out


def sensor(p: Problem, w: np.ndarray):
    w = _state(p, w)
    s = np.zeros(p.shape[1:])
    d = np.zeros(p.shape[1:])
    cfg = p.cfg()
    if lib().or_sensor(C.byref(cfg), _dp(w), _dp(s), _dp(d)):
        raise MemoryError("oracle sensor failed")
    return s, d


def dt(p: Problem, w: np.ndarray, cfl: float) -> float:
    w = _state(p, w)
    cfg = p.cfg()
    return float(lib().or_dt(C.byref(cfg), _dp(w), cfl))


def step(p: Problem, w: np.ndarray, n: int, *, cfl: float = 0.0, dt_fixed: float = 0.0,
         dt_every: int = 1, step0: int = 0, dt0: float = 0.0):
    """n RK3 steps; returns (w_new, step_counter, dt)."""
    w = _state(p, w).copy()
    cfg = p.cfg()
    st = C.c_longlong(step0)
    d = C.c_double(dt0 if dt0 > 0 else dt_fixed)
    if lib().or_step(C.byref(cfg), _dp(w), n, cfl, dt_fixed, dt_every, C.byref(st), C.byref(d)):
        raise MemoryError("oracle step failed")
    return w, int(st.value), float(d.value)


def metric(p: Problem):
    cfg = p.cfg()
    ey = np.zeros(p.ny)
    eyy = np.zeros(p.ny)
    lib().or_metric(C.byref(cfg), _dp(ey), _dp(eyy))
    return ey, eyy


def weno_rec(order: int, f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (order,)
    return float(lib().or_weno_rec(order, _dp(f)))


def weno_parts(order: int, f):
    """Candidate values q_k and smoothness indicators beta_k."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (order,)
    q = np.zeros(4)
    b = np.zeros(4)
    r = lib().or_weno_parts(order, _dp(f), _dp(q), _dp(b))
    return q[:r], b[:r]


def eigvec(gamma: float, direction: int, uvec, H: float):
    u = np.ascontiguousarray(uvec, dtype=np.float64)
    L = np.zeros(25)
    R = np.zeros(25)
    c = lib().or_eigvec(gamma, direction, _dp(u), H, _dp(L), _dp(R))
    return L.reshape(5, 5), R.reshape(5, 5), float(c)


def eigvec_tp(chi: float, c: float, direction: int, uvec, H: float):
    """Eigenvector matrices for a general equation of state (chi = (1/rho)
    dp/de at constant rho, speed of sound c)."""
    u = np.ascontiguousarray(uvec, dtype=np.float64)
    L = np.zeros(25)
    R = np.zeros(25)
    lib().or_eigvec_tp(chi, c, direction, _dp(u), H, _dp(L), _dp(R))
    return L.reshape(5, 5), R.reshape(5, 5)


def thermo(p: Problem, T: float):
    """(c_p, dc_p/dT, e) of the problem's gas at temperature T."""
    cfg = p.cfg()
    cp, dcp, e = C.c_double(), C.c_double(), C.c_double()
    lib().or_thermo(C.byref(cfg), T, C.byref(cp), C.byref(dcp), C.byref(e))
    return cp.value, dcp.value, e.value


def temperature(p: Problem, target: float, enthalpy: bool = False, T0: float = 1.0) -> float:
    """T with e(T) = target (or h(T) = target, Newton from T0)."""
    cfg = p.cfg()
    return float(lib().or_temperature(C.byref(cfg), target, 1 if enthalpy else 0, T0))


def roe_state(p: Problem, a, b):
    """Roe state (u, v, w, H, chi, c) of the WENO flux between the states a
    and b, each (rho, u, v, w, T)."""
    cfg = p.cfg()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(6)
    lib().or_roe_state(C.byref(cfg), _dp(a), _dp(b), _dp(out))
    return out


def conserved(p: Problem, rho, u, v, w, T) -> np.ndarray:
    """State (rho, rho u, rho v, rho w, rho E) of primitive fields, with the
    problem's internal energy e(T) (element by element)."""
    rho, u, v, w, T = [np.asarray(f, dtype=np.float64) for f in (rho, u, v, w, T)]
    shape = np.broadcast(rho, u, v, w, T).shape
    e = np.vectorize(lambda t: thermo(p, float(t))[2], otypes=[np.float64])(T)
    out = np.empty((5,) + shape)
    out[0] = rho
    out[1] = rho * u
    out[2] = rho * v
    out[3] = rho * w
    out[4] = rho * (e + 0.5 * (u * u + v * v + w * w))
    return out


def rk3_scalar(lam: float, y0: float, dt_: float, n: int) -> float:
    return float(lib().or_rk3_scalar(lam, y0, dt_, n))
