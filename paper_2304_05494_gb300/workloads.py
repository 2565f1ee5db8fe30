"""Seeded synthetic inputs shaped like the paper's channel and box workloads.

This module only builds initial states and grids (closed-form fields plus
seeded noise, numpy ``default_rng``); it holds none of the solver's
arithmetic.  Both the CUDA path and the CPU oracle consume its output.

States are float64 arrays of shape (5, nz, ny, nx) holding the conserved
variables (rho, rho u, rho v, rho w, rho E) in reference units: reference
density, velocity, temperature and length 1, gas constant R = 1/(gamma M^2),
E = c_v T + |u|^2 / 2 with c_v = R/(gamma - 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 1234


@dataclass
class Case:
    """A workload: grid, gas, boundaries, scheme and its initial state."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    w0: np.ndarray
    y: Optional[np.ndarray] = None
    gamma: float = 1.4
    prandtl: float = 0.72
    mach: float = 0.1
    re: float = 1600.0
    visc_exp: float = 0.76
    t_ref: float = 1.0
    wall_y: bool = False
    t_wall: float = 1.0
    force: bool = False
    weno_order: int = 0
    threshold: float = 0.2
    cfl: float = 0.8
    dt_fixed: float = 0.0
    dt_every: int = 10
    steps: int = 10
    extra: dict = field(default_factory=dict)
    # the primitive fields (rho, u, v, w, T) w0 was built from, where kept:
    # the same initial flow for another gas model
    prim0: Optional[np.ndarray] = None

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz


def conserved(rho, u, v, w, T, gamma, mach):
    """Conserved variables of a calorically perfect gas in reference units."""
    R = 1.0 / (gamma * mach * mach)
    cv = R / (gamma - 1.0)
    E = cv * T + 0.5 * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, rho * E]), dtype=np.float64)


def taylor_green(n: int = 32, mach: float = 0.1, re: float = 1600.0, seed: int = SEED_BASE + 0,
                 noise: float = 1e-6) -> Case:
    """Taylor-Green vortex on the triply periodic [0, 2 pi]^3 box: closed-form
    velocity and pressure, T = 1, density p/(R T) times (1 + noise xi),
    xi ~ U(-1, 1) seeded."""
    L = 2.0 * np.pi
    x = np.arange(n) * (L / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    gamma = 1.4
    R = 1.0 / (gamma * mach * mach)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p0 = R  # rho0 R T0
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    T = np.ones_like(u)
    rng = np.random.default_rng(seed)
    rho = p / (R * T) * (1.0 + noise * rng.uniform(-1.0, 1.0, size=u.shape))
    w0 = conserved(rho, u, v, w, T, gamma, mach)
    return Case("taylor_green_%d" % n, n, n, n, L, L, L, w0, gamma=gamma, mach=mach, re=re,
                visc_exp=0.76, prandtl=0.72, weno_order=0, cfl=0.8, steps=10)


def tanh_nodes(ny: int, beta: float) -> np.ndarray:
    """Cell-centre nodes of a channel of half height 1 clustered at the
    walls y = -1, +1: y = tanh(beta xi)/tanh(beta), xi = -1 + (j + 1/2) 2/ny."""
    xi = -1.0 + (np.arange(ny) + 0.5) * 2.0 / ny
    return np.tanh(beta * xi) / np.tanh(beta)


def tanh_beta_for(ny: int, dy_wall: float) -> float:
    """Stretching parameter whose first cell (wall to the mirror face of the
    first node, i.e. twice the first node's wall distance) equals dy_wall."""
    lo, hi = 1e-6, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        d = 2.0 * (tanh_nodes(ny, mid)[0] + 1.0)
        if d > dy_wall:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _smooth_noise(rng, kmax_xz: int, kmax_y: int, x, y, z, lx, lz):
    """Sum of random-amplitude, random-phase separable Fourier modes
    cos(kx x + a) sin(ky pi (y+1)/2 + b) cos(kz z + c), max-normalised;
    returned with shape (nz, ny, nx)."""
    cx, sy, cz, amp = [], [], [], []
    for kx in range(0, kmax_xz + 1):
        for kz in range(0, kmax_xz + 1):
            if kx == 0 and kz == 0:
                continue
            for ky in range(1, kmax_y + 1):
                amp.append(rng.normal())
                ph = rng.uniform(0, 2 * np.pi, size=3)
                cx.append(np.cos(2 * np.pi * kx * x / lx + ph[0]))
                cz.append(np.cos(2 * np.pi * kz * z / lz + ph[1]))
                sy.append(np.sin(0.5 * np.pi * ky * (y + 1.0) + ph[2]))
    a = np.asarray(amp)[:, None] * np.asarray(cz)
    g = np.einsum("mk,mj,mi->kji", a, np.asarray(sy), np.asarray(cx), optimize=True)
    return g / np.max(np.abs(g))


def channel(nx: int = 256, ny: int = 128, nz: int = 128, mach_b: float = 1.5, re_b: float = 3000.0,
            re_tau: float = 220.0, dy_plus_wall: float = 0.7, amp: float = 0.1,
            seed: int = SEED_BASE + 1, weno_order: int = 5, kmax_xz: int = 6, kmax_y: int = 4) -> Case:
    """Compressible channel, bulk Mach 1.5, 6 pi h x 2h x 2 pi h, tanh nodes
    in y with the first wall cell at dy+_wall, isothermal no-slip walls at
    T_w = 1, periodic x/z.  Laminar Poiseuille profile u = 3/2 (1 - y^2)
    (bulk velocity 1) with rho = T = 1, plus seeded smooth random velocity
    perturbations of amplitude amp (random-phase Fourier modes, damped by
    (1 - y^2) towards the walls).  Re_b = 3000 with the wall viscosity gives
    Re_tau ~ 220 for this Mach number (Coleman, Kim & Moser 1995)."""
    lx, ly, lz = 6.0 * np.pi, 2.0, 2.0 * np.pi
    beta = tanh_beta_for(ny, dy_plus_wall / re_tau)
    yn = tanh_nodes(ny, beta)
    x = np.arange(nx) * (lx / nx)
    z = np.arange(nz) * (lz / nz)
    rng = np.random.default_rng(seed)
    damp = (1.0 - yn * yn)[None, :, None]
    u = 1.5 * damp + amp * damp * _smooth_noise(rng, kmax_xz, kmax_y, x, yn, z, lx, lz)
    v = amp * damp * _smooth_noise(rng, kmax_xz, kmax_y, x, yn, z, lx, lz)
    w = amp * damp * _smooth_noise(rng, kmax_xz, kmax_y, x, yn, z, lx, lz)
    rho = np.ones_like(u)
    T = np.ones_like(u)
    w0 = conserved(rho, u, v, w, T, 1.4, mach_b)
    return Case("channel_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, lx, ly, lz, w0, y=yn, gamma=1.4,
                mach=mach_b, re=re_b, visc_exp=0.76, prandtl=0.72, wall_y=True, t_wall=1.0,
                force=True, weno_order=weno_order, threshold=0.2, cfl=0.8, steps=200,
                extra={"beta": beta, "re_tau": re_tau},
                prim0=np.ascontiguousarray(np.stack([rho, u, v, w, T]), dtype=np.float64))


def smooth_periodic(nx: int, ny: int, nz: int, seed: int, mach: float = 0.5, amp_u: float = 0.5,
                    amp_s: float = 0.1, kmax: int = 3, lx: float = 2 * np.pi, ly: float = 2 * np.pi,
                    lz: float = 2 * np.pi):
    """Random smooth periodic (rho, u, v, w, T): a few seeded Fourier modes;
    rho and T positive around 1.  Returns the conserved state."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny)
    z = np.arange(nz) * (lz / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")

    def field_(amp):
        g = np.zeros(X.shape)
        for _ in range(6):
            k = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.normal()
            g += a * np.cos(2 * np.pi * (k[0] * X / lx + k[1] * Y / ly + k[2] * Z / lz) + ph)
        return amp * g / max(np.max(np.abs(g)), 1e-30)

    rho = 1.0 + field_(amp_s)
    T = 1.0 + field_(amp_s)
    u, v, w = field_(amp_u), field_(amp_u), field_(amp_u)
    return conserved(rho, u, v, w, T, 1.4, mach)


def isentropic_vortex(n: int, beta: float = 5.0, L: float = 10.0, nz: int = 1):
    """Shu's isentropic vortex on the periodic [0, L]^2 (x thin z), free
    stream rho = u = v = p = 1, so R = 1 (Mach parameter 1/sqrt(gamma)) and
    T = p/rho.  Returns (conserved state, mach parameter)."""
    gamma = 1.4
    mach = 1.0 / np.sqrt(gamma)
    x = (np.arange(n) + 0.5) * (L / n)
    z = np.arange(nz) * 1.0
    Z, Y, X = np.meshgrid(z, x, x, indexing="ij")
    xb, yb = X - 0.5 * L, Y - 0.5 * L
    r2 = xb * xb + yb * yb
    du = -beta / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * yb
    dv = beta / (2 * np.pi) * np.exp(0.5 * (1 - r2)) * xb
    T = 1.0 - (gamma - 1.0) * beta * beta / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return conserved(rho, 1.0 + du, 1.0 + dv, np.zeros_like(T), T, gamma, mach), mach


def double_sod(n: int, L: float = 2.0):
    """Two mirrored Sod problems on the periodic [0, L): high state
    (rho, p) = (1, 1) on [L/4, 3L/4), low state (0.125, 0.1) elsewhere, at
    rest; R = 1.  Returns (conserved state shaped (5, 1, 1, n), cell
    centres, mach parameter)."""
    gamma = 1.4
    mach = 1.0 / np.sqrt(gamma)
    x = (np.arange(n) + 0.5) * (L / n)
    hi = (x >= 0.25 * L) & (x < 0.75 * L)
    rho = np.where(hi, 1.0, 0.125)
    p = np.where(hi, 1.0, 0.1)
    T = p / rho
    z = np.zeros_like(x)
    w0 = conserved(rho, z, z, z, T, gamma, mach).reshape(5, 1, 1, n)
    return np.ascontiguousarray(w0), x, mach


def isotropic(n: int = 512, mach_t: float = 0.6, re_lambda: float = 100.0, k0: float = 4.0,
              seed: int = SEED_BASE + 2, weno_order: int = 7) -> Case:
    """Decaying compressible isotropic turbulence on the periodic [0, 2 pi]^3:
    a seeded random-phase solenoidal velocity with energy spectrum
    E(k) ~ k^4 exp(-2 (k/k0)^2), scaled to the turbulent Mach number
    M_t = sqrt(<u.u>)/c = mach_t, with uniform density and temperature
    (rho = T = 1, reference Mach 1 so that c = 1).  Re follows from
    Re_lambda = u' lambda / nu with u' = sqrt(<u.u>/3) and the Taylor
    microscale of the initial spectrum."""
    L = 2.0 * np.pi
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kk[0, 0, 0] = 1.0
    # random complex vector field, projected onto the solenoidal subspace
    comps = [rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape) for _ in range(3)]
    kdot = (kx * comps[0] + ky * comps[1] + kz * comps[2]) / (kk * kk)
    comps = [comps[0] - kx * kdot, comps[1] - ky * kdot, comps[2] - kz * kdot]
    amp = np.sqrt(kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2) / (4.0 * np.pi * kk * kk))
    amp[0, 0, 0] = 0.0
    vel = []
    for c in comps:
        f = np.fft.ifftn(c * amp).real
        vel.append(f)
    del comps, kdot
    u2 = np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    gamma = 1.4
    mach_ref = 1.0
    c0 = 1.0 / mach_ref  # sound speed at T = 1 in reference units
    scale = mach_t * c0 / np.sqrt(u2)
    vel = [v * scale for v in vel]
    # Taylor microscale from the discrete velocity gradient
    dudx = np.gradient(vel[0], L / n, axis=2)
    uprime = np.sqrt(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) / 3.0)
    lam = uprime / np.sqrt(np.mean(dudx * dudx))
    del dudx
    re = re_lambda / (uprime * lam)  # nu = 1/Re at rho = T = 1
    one = np.ones_like(vel[0])
    w0 = conserved(one, vel[0], vel[1], vel[2], one, gamma, mach_ref)
    return Case("isotropic_%d" % n, n, n, n, L, L, L, w0, gamma=gamma, mach=mach_ref, re=re,
                visc_exp=0.76, prandtl=0.72, weno_order=weno_order, threshold=0.2, cfl=0.8, steps=100,
                extra={"mach_t": mach_t, "re_lambda": re_lambda, "uprime": uprime, "lambda": lam})


def channel_big(seed: int = SEED_BASE + 3, weno_order: int = 5) -> Case:
    """The large channel: 1024 x 256 x 512 points on 6 pi h x 2h x 2 pi h,
    Re_tau ~ 550 (Re_b ~ 8400 on the wall viscosity, scaled from the
    Re_b = 3000 / Re_tau = 222 pair of the M = 1.5 channel with the
    Re_tau ~ Re_b^0.88 law), first wall cell at dy+ = 0.7."""
    re_b = 3000.0 * (550.0 / 222.0) ** (1.0 / 0.88)
    c = channel(1024, 256, 512, re_b=re_b, re_tau=550.0, seed=seed, weno_order=weno_order)
    c.name = "channel_1024x256x512"
    c.steps = 100
    return c
