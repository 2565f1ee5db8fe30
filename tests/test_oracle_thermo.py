"""Pins of the oracle's thermally perfect gas (paper Sec. 2: specific heats
depending on temperature through NASA polynomials).

The gas: c_p/R = sum_{l=-2..4} a_l T^l (the NASA Glenn 9-coefficient form in
reference units of T).  Each check compares the oracle with something other
than its own formulas: quadrature and numerical differentiation of the
polynomial, root finding, the numerical Jacobian of the Euler flux under
this equation of state, the calorically perfect oracle (a constant
polynomial), discrete invariants, and an analytic right-hand side built by
sympy, whose own integration supplies e(T).
"""
import numpy as np
import pytest
import sympy as sp
from scipy import integrate, optimize

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W

GAMMA = 1.4
# A synthetic gas whose gamma falls from 1.45 at T = 0.5 through 1.40 at
# T = 1 to 1.35 at T = 2 (air-like trend), with every kind of term, the
# T^-2 and the logarithmic T^-1 ones included.
A_TP = np.array([0.05, -0.2, 3.2, 0.5, -0.06, 0.004, 0.0])
A_CONST = np.array([0.0, 0.0, GAMMA / (GAMMA - 1.0), 0.0, 0.0, 0.0, 0.0])


def _cp_over_r(a, T):
    return sum(a[l + 2] * T ** l for l in range(-2, 5))


def _prob(nx, ny, nz, L=2 * np.pi, **kw):
    return O.Problem(nx, ny, nz, L, L, L, **kw)


def test_energy_is_the_integral_of_cv():
    """e(T2) - e(T1) = int c_v dT (quadrature), c_p the polynomial, dc_p/dT
    its numerical derivative; a constant polynomial gives e = c_v T."""
    mach = 0.5
    R = 1.0 / (GAMMA * mach ** 2)
    p = _prob(4, 4, 4, mach=mach, cp_coef=A_TP)
    for T1, T2 in ((0.4, 1.0), (1.0, 2.7), (0.8, 1.3)):
        de = O.thermo(p, T2)[2] - O.thermo(p, T1)[2]
        quad, _ = integrate.quad(lambda t: R * (_cp_over_r(A_TP, t) - 1.0), T1, T2, epsabs=0, epsrel=2e-14)
        assert abs(de - quad) < 1e-12 * abs(quad)
    for T in (0.5, 1.0, 1.9):
        cp, dcp, _ = O.thermo(p, T)
        assert abs(cp - R * _cp_over_r(A_TP, T)) < 1e-14 * cp
        h = 1e-4 * T
        num = (O.thermo(p, T + h)[0] - O.thermo(p, T - h)[0]) / (2 * h)
        assert abs(dcp - num) < 1e-7 * abs(num)
    pc = _prob(4, 4, 4, mach=mach, cp_coef=A_CONST)
    for T in (0.3, 1.0, 2.5):
        cp, dcp, e = O.thermo(pc, T)
        assert abs(e - R / (GAMMA - 1.0) * T) < 1e-14 * e
        assert abs(cp - GAMMA * R / (GAMMA - 1.0)) < 1e-14 * cp and dcp == 0.0


def test_temperature_inverts_energy_and_enthalpy():
    """The primitive recovery's inversion of e(T) and the Roe state's
    inversion of h(T) = e + R T agree with a bracketing root finder."""
    mach = 0.7
    R = 1.0 / (GAMMA * mach ** 2)
    p = _prob(4, 4, 4, mach=mach, cp_coef=A_TP)
    for T in (0.35, 0.9, 1.0, 1.6, 3.0):
        e = O.thermo(p, T)[2]
        ref = optimize.brentq(lambda t: O.thermo(p, t)[2] - e, 0.2, 5.0, xtol=1e-15, rtol=1e-15)
        assert abs(O.temperature(p, e) - ref) < 2e-15 * ref
        assert abs(O.temperature(p, e + R * T, enthalpy=True, T0=1.3 * T) - T) < 2e-15 * T


def _tp_flux(p, U, d):
    """Euler flux of the conserved state U under the thermally perfect
    equation of state p = rho R T(e), T from a bracketing root finder."""
    R = 1.0 / (p.gamma * p.mach ** 2)
    rho, m, E = U[0], U[1:4], U[4]
    u = m / rho
    e = E / rho - 0.5 * np.dot(u, u)
    T = optimize.brentq(lambda t: O.thermo(p, t)[2] - e, 0.05, 20.0, xtol=1e-15, rtol=1e-15)
    pr = rho * R * T
    F = np.empty(5)
    F[0] = m[d]
    F[1:4] = m[d] * u
    F[1 + d] += pr
    F[4] = (E + pr) * u[d]
    return F


@pytest.mark.parametrize("d", [0, 1, 2])
def test_eigenvectors_diagonalise_the_thermally_perfect_jacobian(d):
    """At a single state the Roe state is that state; its chi and c make
    L R = I and L A R = diag(u-c, u, u, u, u+c), A = dF/dU by central
    differences of the flux under the thermally perfect equation of state
    (pins c^2 = gamma(T) R T, chi = R/c_v(T) and the entropy-wave column)."""
    mach = 0.6
    p = _prob(4, 4, 4, mach=mach, cp_coef=A_TP)
    rng = np.random.default_rng(40 + d)
    for _ in range(2):
        rho, T = rng.uniform(0.6, 1.8), rng.uniform(0.6, 2.2)
        u = rng.normal(size=3)
        st = np.array([rho, *u, T])
        roe = O.roe_state(p, st, st)
        assert np.allclose(roe[:3], u, rtol=0, atol=1e-15)
        L, Rm = O.eigvec_tp(roe[4], roe[5], d, roe[:3], roe[3])
        assert np.allclose(L @ Rm, np.eye(5), atol=1e-12)
        E = rho * (O.thermo(p, T)[2] + 0.5 * np.dot(u, u))
        U = np.array([rho, *(rho * u), E])
        A = np.zeros((5, 5))
        for k in range(5):
            h = 1e-5 * max(abs(U[k]), 1.0)
            Up, Um = U.copy(), U.copy()
            Up[k] += h
            Um[k] -= h
            A[:, k] = (_tp_flux(p, Up, d) - _tp_flux(p, Um, d)) / (2 * h)
        lam = L @ A @ Rm
        c = roe[5]
        expect = np.diag([u[d] - c, u[d], u[d], u[d], u[d] + c])
        assert np.allclose(lam, expect, atol=2e-7 * (abs(u[d]) + c)), lam - expect
        # gamma changes with T: the sound speed is not the reference gamma's
        R = 1.0 / (GAMMA * mach ** 2)
        assert abs(c - np.sqrt(GAMMA * R * T)) > 1e-4 * c or abs(T - 1.0) < 0.05


def test_roe_state_of_two_states():
    """Two different states: L R = I at their Roe state, H~ the sqrt(rho)
    weighted total enthalpy, and h(T~) = H~ - |u~|^2/2."""
    mach = 0.6
    R = 1.0 / (GAMMA * mach ** 2)
    p = _prob(4, 4, 4, mach=mach, cp_coef=A_TP)
    a = np.array([1.3, 0.4, -0.2, 0.1, 0.8])
    b = np.array([0.7, -0.3, 0.5, 0.2, 1.9])
    roe = O.roe_state(p, a, b)
    wa, wb = np.sqrt(a[0]), np.sqrt(b[0])
    Ha = O.thermo(p, a[4])[2] + R * a[4] + 0.5 * np.dot(a[1:4], a[1:4])
    Hb = O.thermo(p, b[4])[2] + R * b[4] + 0.5 * np.dot(b[1:4], b[1:4])
    assert abs(roe[3] - (wa * Ha + wb * Hb) / (wa + wb)) < 1e-14 * roe[3]
    ht = roe[3] - 0.5 * np.dot(roe[:3], roe[:3])
    Tt = optimize.brentq(lambda t: O.thermo(p, t)[2] + R * t - ht, 0.1, 10.0, xtol=1e-15, rtol=1e-15)
    cp = O.thermo(p, Tt)[0]
    assert abs(roe[4] - R / (cp - R)) < 1e-13 * roe[4]
    assert abs(roe[5] - np.sqrt(cp / (cp - R) * R * Tt)) < 1e-13 * roe[5]
    L, Rm = O.eigvec_tp(roe[4], roe[5], 1, roe[:3], roe[3])
    assert np.allclose(L @ Rm, np.eye(5), atol=1e-12)


def test_constant_polynomial_is_the_calorically_perfect_gas():
    """c_p/R = gamma/(gamma-1) through the thermally perfect code (Newton
    inversions, general eigenvectors, c_p(T) in the heat flux) reproduces
    the calorically perfect oracle: same WENO flags, right-hand side and dt
    to round-off, on a walled channel with WENO, viscosity and forcing."""
    c = W.channel(16, 20, 8, seed=3)
    kw = dict(y=c.y, wall_y=True, mach=c.mach, re=c.re, force=True, weno_order=5, threshold=0.05)
    pc = O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, **kw)
    pt = O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, cp_coef=A_CONST, **kw)
    rc, fc = O.rhs(pc, c.w0, flags=True)
    rt, ft = O.rhs(pt, c.w0, flags=True)
    frac = np.mean(np.concatenate([f.ravel() for f in fc]))
    assert 0.02 < frac < 0.98
    for a, b in zip(fc, ft):
        assert np.array_equal(a, b)
    err = np.max(np.abs(rt - rc), axis=(1, 2, 3)) / np.max(np.abs(rc), axis=(1, 2, 3))
    assert np.all(err < 1e-12), err
    assert abs(O.dt(pt, c.w0, 0.8) - O.dt(pc, c.w0, 0.8)) < 1e-14 * O.dt(pc, c.w0, 0.8)


@pytest.mark.parametrize("weno", [0, 5, 7])
def test_thermally_perfect_free_stream_and_conservation(weno):
    """A uniform state has R = 0 (inviscid exactly), uniform and stretched
    y; on a periodic box every inviscid R sums to round-off with WENO on
    part of the interfaces."""
    xi = np.arange(14) * 2 * np.pi / 14
    y = xi + 0.25 * np.sin(xi)
    p = _prob(10, 14, 9, y=y, mach=0.6, re=50.0, weno_order=weno, threshold=-1.0, cp_coef=A_TP)
    one = np.ones((9, 14, 10))
    w = O.conserved(p, 1.2 * one, 0.3 * one, -0.2 * one, 0.1 * one, 1.7 * one)
    assert np.max(np.abs(O.rhs(p, w, terms=O.CONV))) == 0.0
    assert np.max(np.abs(O.rhs(p, w))) < 1e-13
    p2 = _prob(12, 14, 10, y=y, mach=0.6, re=-1.0, weno_order=weno, threshold=0.3, cp_coef=A_TP)
    w2 = W.smooth_periodic(12, 14, 10, seed=5, mach=0.6, amp_u=0.8, amp_s=0.3)
    r, flags = O.rhs(p2, w2, flags=True)
    if weno:
        frac = np.mean(np.concatenate([f.ravel() for f in flags]))
        assert 0.05 < frac < 0.95
    ey, _ = O.metric(p2)
    dv = (1.0 / ey)[None, None, :, None]
    tot = np.sum(r * dv, axis=(1, 2, 3))
    scale = np.sum(np.abs(r) * dv, axis=(1, 2, 3))
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_thermally_perfect_quiescent_walls_fixed_point():
    """Quiescent gas at the wall temperature between isothermal walls is a
    fixed point of the whole RHS (WENO everywhere, viscous, forced)."""
    y = W.tanh_nodes(16, 1.5)
    p = O.Problem(8, 16, 6, 3.0, 2.0, 2.0, y=y, wall_y=True, t_wall=1.6, mach=1.5, re=300.0,
                  weno_order=5, threshold=-1.0, force=True, cp_coef=A_TP)
    one = np.ones((6, 16, 8))
    w = O.conserved(p, 0.9 * one, 0 * one, 0 * one, 0 * one, 1.6 * one)
    # T comes back from e by Newton's method to within an ulp of T_w, so
    # the mirrored ghosts match to round-off rather than exactly
    assert np.max(np.abs(O.rhs(p, w, terms=O.CONV))) < 1e-14
    assert np.max(np.abs(O.rhs(p, w))) < 1e-12


def _tp_rhs_exact(fields, mach, re, pr, visc_exp, a):
    """Analytic Navier-Stokes RHS of closed-form (rho, u, v, w, T) for the
    thermally perfect gas: e(T) by sympy's integration of c_v, h = e + R T,
    k = mu c_p(T) / Pr.  Returns the lambdified fields, E and the RHS."""
    x, y, z, t = sp.symbols("x y z t")
    rho, u, v, w, T = fields
    R = 1 / (GAMMA * sp.nsimplify(mach) ** 2)
    ar = [sp.nsimplify(c) for c in a]
    cp_t = R * sum(ar[l + 2] * t ** l for l in range(-2, 5))
    e_t = sp.integrate(cp_t - R, t)
    cp = cp_t.subs(t, T)
    e = e_t.subs(t, T)
    p = rho * R * T
    U = [u, v, w]
    X = [x, y, z]
    H = e + R * T + (u * u + v * v + w * w) / 2
    mu = T ** sp.nsimplify(visc_exp) / re
    kc = mu * cp / pr
    th = sum(sp.diff(U[q], X[q]) for q in range(3))
    tau = [[mu * (sp.diff(U[q], X[b]) + sp.diff(U[b], X[q]) - (sp.Rational(2, 3) * th if q == b else 0))
            for b in range(3)] for q in range(3)]
    out = [-sum(sp.diff(rho * U[j], X[j]) for j in range(3))]
    for i in range(3):
        out.append(-sum(sp.diff(rho * U[i] * U[j] + (p if i == j else 0), X[j]) for j in range(3))
                   + sum(sp.diff(tau[i][j], X[j]) for j in range(3)))
    out.append(-sum(sp.diff(rho * U[j] * H, X[j]) for j in range(3))
               + sum(sp.diff(sum(U[i] * tau[i][j] for i in range(3)) + kc * sp.diff(T, X[j]), X[j])
                     for j in range(3)))
    E = rho * (e + (u * u + v * v + w * w) / 2)
    f = [sp.lambdify((x, y, z), q, "numpy") for q in fields]
    fe = sp.lambdify((x, y, z), E, "numpy")
    r = [sp.lambdify((x, y, z), q, "numpy") for q in out]
    return f, fe, r


@pytest.mark.parametrize("stretched", [False, True])
def test_thermally_perfect_design_order_manufactured(stretched):
    """R_h(w*) - R(w*) falls at 6th order for the central split-form flux
    plus the Laplacian-form viscous terms with c_p(T) in the heat flux, T
    spanning 0.7 .. 1.3 (gamma varies by ~3%)."""
    x, y, z = sp.symbols("x y z")
    rho = 1 + sp.Rational(1, 5) * sp.sin(x + sp.Rational(3, 10)) * sp.cos(y) + sp.sin(z) / 10
    u = sp.sin(y + z) / 2 + sp.cos(x) / 5
    v = sp.Rational(2, 5) * sp.cos(x + z) - sp.sin(y) / 10
    w = sp.Rational(3, 10) * sp.sin(x - y) + sp.cos(z) / 5
    T = 1 + sp.cos(x) * sp.sin(y + z) * sp.Rational(3, 10)
    mach, re = 0.5, 100.0
    f, fe, rhs = _tp_rhs_exact((rho, u, v, w, T), mach, re, 0.72, 0.76, A_TP)
    errs = []
    for n in (16, 32):
        xi = np.arange(n) * 2 * np.pi / n
        yv = xi + 0.3 * np.sin(xi) if stretched else xi
        Z, Y, X = np.meshgrid(xi, yv, xi, indexing="ij")
        vals = [g(X, Y, Z) * np.ones_like(X) for g in f]
        wv = np.stack([vals[0], vals[0] * vals[1], vals[0] * vals[2], vals[0] * vals[3],
                       fe(X, Y, Z) * np.ones_like(X)])
        p = _prob(n, n, n, y=yv if stretched else None, mach=mach, re=re, prandtl=0.72, visc_exp=0.76,
                  weno_order=0, cp_coef=A_TP)
        r = O.rhs(p, wv)
        ex = np.stack([g(X, Y, Z) * np.ones_like(X) for g in rhs])
        errs.append(np.max(np.abs(r - ex), axis=(1, 2, 3)) / np.max(np.abs(ex), axis=(1, 2, 3)))
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > 5.4), rates


def test_thermally_perfect_design_order_with_walls():
    """Isothermal no-slip walls with the thermally perfect gas: fields whose
    mirror continuation is analytic (velocity and T - T_w odd about each
    wall, pressure even) converge at 6th order, wall rows included -- this
    pins the wall ghosts' rho = p/(R T) and H = h(T) + |u|^2/2 with h(T)
    from the polynomial."""
    x, y, z = sp.symbols("x y z")
    mach, tw = 0.8, 1.0
    R = 1 / (GAMMA * sp.nsimplify(mach) ** 2)
    cy, sy = sp.cos(sp.pi * y / 2), sp.sin(sp.pi * y)
    u = (sp.Rational(3, 2) + sp.sin(x + z) / 5) * cy
    v = sp.Rational(3, 10) * sy * sp.cos(x)
    w = sp.Rational(2, 5) * cy * sp.sin(z)
    T = tw + sp.Rational(3, 10) * cy * (1 + sp.cos(x) / 10)
    p = R * (1 + sp.cos(sp.pi * y) * sp.cos(z) / 10)
    rho = p / (R * T)
    f, fe, rhs = _tp_rhs_exact((rho, u, v, w, T), mach, 50.0, 0.72, 0.76, A_TP)
    errs = []
    for ny in (16, 32):
        nx = nz = ny // 2
        xs = np.arange(nx) * 2 * np.pi / nx
        zs = np.arange(nz) * 2 * np.pi / nz
        ys = -1.0 + (np.arange(ny) + 0.5) * 2.0 / ny
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        vals = [g(X, Y, Z) * np.ones_like(X) for g in f]
        wv = np.stack([vals[0], vals[0] * vals[1], vals[0] * vals[2], vals[0] * vals[3],
                       fe(X, Y, Z) * np.ones_like(X)])
        pr = O.Problem(nx, ny, nz, 2 * np.pi, 2.0, 2 * np.pi, wall_y=True, t_wall=tw, mach=mach, re=50.0,
                       weno_order=0, cp_coef=A_TP)
        r = O.rhs(pr, wv)
        ex = np.stack([g(X, Y, Z) * np.ones_like(X) for g in rhs])
        errs.append(np.max(np.abs(r - ex), axis=(1, 2, 3)) / np.max(np.abs(ex), axis=(1, 2, 3)))
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > 5.0), rates


def test_thermally_perfect_dt_closed_form_uniform():
    """CFL dt of a uniform state: c = sqrt(gamma(T) R T) and the viscous
    term gamma(T) mu / (Pr rho), gamma(T) = c_p/(c_p - R) of the polynomial."""
    mach, T, rho = 0.5, 1.7, 1.3
    R = 1.0 / (GAMMA * mach ** 2)
    p = _prob(8, 8, 8, mach=mach, re=200.0, prandtl=0.7, cp_coef=A_TP)
    one = np.ones((8, 8, 8))
    w = O.conserved(p, rho * one, 0.4 * one, -0.3 * one, 0.2 * one, T * one)
    cp = R * _cp_over_r(A_TP, T)
    gam = cp / (cp - R)
    c = np.sqrt(gam * R * T)
    h = 2 * np.pi / 8
    conv = (0.4 + c + 0.3 + c + 0.2 + c) / h
    visc = gam * (T ** 0.76 / 200.0) / (0.7 * rho) * 3 / h ** 2
    assert abs(O.dt(p, w, 0.8) - 0.8 / (conv + visc)) < 1e-13 * (0.8 / (conv + visc))
    # and gamma(T) is not the reference gamma here
    assert abs(gam - GAMMA) > 1e-3
