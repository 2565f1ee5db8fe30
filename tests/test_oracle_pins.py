"""Pins of the CPU oracle against facts fixed by mathematics and published
methods (closed forms, invariants, exact solutions, convergence orders).

None of these recomputes an oracle formula the same way; each checks a
property that a dropped term, a wrong sign, index or coefficient breaks.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_2304_05494_gb300 import workloads as W
from tests import exact_riemann as ER

A1 = (0.75, -0.15, 1.0 / 60.0)
# Taylor-series coefficients of the central first derivative of orders 2..8,
# derived here by solving the moment conditions (not read from the oracle)
def central_coeffs(order):
    L = order // 2
    # sum_l a_l 2 l^(2m-1) = delta_{m1}, m = 1..L
    M = np.array([[2.0 * l ** (2 * m - 1) for l in range(1, L + 1)] for m in range(1, L + 1)])
    rhs = np.zeros(L)
    rhs[0] = 1.0
    return tuple(np.linalg.solve(M, rhs))


def mod_wavenumber(k, h, order=6):
    """Closed form of the central first derivative of this order on exp(ikx)."""
    a = central_coeffs(order)
    return 2.0 * sum(c * np.sin((l + 1) * k * h) for l, c in enumerate(a)) / h


def _prob(nx, ny, nz, L=2 * np.pi, **kw):
    return O.Problem(nx, ny, nz, L, L, L, **kw)


# ------------------------------------------------------------------ WENO ---
def _cell_avg_poly(coefs, j):
    """Cell average over [j-1/2, j+1/2] of sum c_n x^n."""
    x = sp.Symbol("x")
    P = sum(c * x ** n for n, c in enumerate(coefs))
    return float(sp.integrate(P, (x, j - sp.Rational(1, 2), j + sp.Rational(1, 2))))


@pytest.mark.parametrize("order,deg", [(3, 1), (5, 2), (7, 3)])
def test_weno_exact_on_polynomials(order, deg):
    """Every substencil reconstructs a polynomial of degree r-1 exactly from
    its cell averages, so any convex weighting returns P(x_{i+1/2})."""
    rng = np.random.default_rng(7)
    r = (order + 1) // 2
    for _ in range(5):
        c = rng.normal(size=deg + 1)
        f = np.array([_cell_avg_poly(c, j) for j in range(-(r - 1), r)])
        exact = sum(cn * 0.5 ** n for n, cn in enumerate(c))
        assert abs(O.weno_rec(order, f) - exact) < 1e-12 * (1 + abs(exact))
        q, _ = O.weno_parts(order, f)
        assert np.allclose(q, exact, atol=1e-12, rtol=0)


def _jiang_shu_reference(order):
    """q_k, beta_k (Jiang-Shu integral definition) and the optimal weights
    derived symbolically from polynomial reconstruction."""
    r = (order + 1) // 2
    x = sp.Symbol("x")
    fs = sp.symbols("f0:%d" % order)
    pts = list(range(-(r - 1), r))
    qs, bs = [], []
    for k in range(r):
        st = pts[k:k + r]
        cs = sp.symbols("c0:%d" % r)
        P = sum(cs[n] * x ** n for n in range(r))
        eqs = [sp.integrate(P, (x, j - sp.Rational(1, 2), j + sp.Rational(1, 2))) - fs[pts.index(j)] for j in st]
        sol = sp.solve(eqs, cs)
        Pk = P.subs(sol)
        qs.append(sp.expand(Pk.subs(x, sp.Rational(1, 2))))
        beta = sum(sp.integrate(sp.diff(Pk, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
                   for l in range(1, r))
        bs.append(sp.expand(beta))
    # big stencil polynomial -> optimal weights
    cs = sp.symbols("C0:%d" % order)
    P = sum(cs[n] * x ** n for n in range(order))
    eqs = [sp.integrate(P, (x, j - sp.Rational(1, 2), j + sp.Rational(1, 2))) - fs[pts.index(j)] for j in pts]
    big = sp.expand(P.subs(sp.solve(eqs, cs)).subs(x, sp.Rational(1, 2)))
    ds = sp.symbols("d0:%d" % r)
    comb = sp.expand(sum(ds[k] * qs[k] for k in range(r)) - big)
    dsol = sp.solve([comb.coeff(f) for f in fs], ds)
    return fs, qs, bs, [dsol[d] for d in ds]


@pytest.mark.parametrize("order", [3, 5, 7])
def test_weno_smoothness_indicators_and_weights(order):
    """beta_k equal the Jiang-Shu integral definition; q_k the substencil
    polynomials; optimal weights reproduce the full-stencil reconstruction
    and give the classic upwind-5 formula (2,-13,47,27,-3)/60 for WENO5."""
    fs, qs, bs, d = _jiang_shu_reference(order)
    if order == 3:
        assert [sp.nsimplify(v) for v in d] == [sp.Rational(1, 3), sp.Rational(2, 3)]
    elif order == 5:
        assert [sp.nsimplify(v) for v in d] == [sp.Rational(1, 10), sp.Rational(3, 5), sp.Rational(3, 10)]
        lin = sp.expand(sum(d[k] * qs[k] for k in range(3)))
        assert [lin.coeff(f) for f in fs] == [sp.Rational(c, 60) for c in (2, -13, 47, 27, -3)]
    else:
        assert [sp.nsimplify(v) for v in d] == [sp.Rational(1, 35), sp.Rational(12, 35),
                                                 sp.Rational(18, 35), sp.Rational(4, 35)]
    rng = np.random.default_rng(3)
    for _ in range(10):
        f = rng.normal(size=order)
        sub = dict(zip(fs, f))
        q, b = O.weno_parts(order, f)
        qref = np.array([float(e.subs(sub)) for e in qs])
        # the Balsara-Shu WENO7 indicators are the integrals scaled by 240
        scale = 240.0 if order == 7 else 1.0
        bref = np.array([float(e.subs(sub)) for e in bs]) * scale
        assert np.allclose(q, qref, rtol=1e-12, atol=1e-12)
        assert np.allclose(b, bref, rtol=1e-10, atol=1e-10)


def test_weno1_is_first_order_upwind():
    """Order 1: the upwind cell value itself."""
    for v in (0.3, -2.0, 7.5):
        assert O.weno_rec(1, [v]) == v


@pytest.mark.parametrize("order,min_rate", [(3, 2.7), (5, 4.5), (7, 6.0)])
def test_weno_convergence_smooth(order, min_rate):
    """On cell averages of a smooth function away from critical points the
    reconstruction converges at the design order."""
    errs = []
    for h in (0.1, 0.05):
        x0 = 0.3  # interface position; sin has no critical point near it
        r = (order + 1) // 2
        centres = x0 - 0.5 * h + h * np.arange(-(r - 1), r)
        f = (np.cos(centres - 0.5 * h) - np.cos(centres + 0.5 * h)) / h  # averages of sin
        errs.append(abs(O.weno_rec(order, f) - np.sin(x0)))
    assert np.log2(errs[0] / errs[1]) > min_rate


def test_weno_non_oscillatory_at_step():
    """At a discontinuity the stencils that cross it get vanishing weight:
    the result stays within the smooth side's range (ENO property)."""
    f = np.array([1.0, 1.0, 1.0, 0.0, 0.0])  # jump between i and i+1
    v = O.weno_rec(5, f)
    assert abs(v - 1.0) < 1e-6
    f7 = np.array([1.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    assert abs(O.weno_rec(7, f7) - 1.0) < 1e-6


# ------------------------------------------------------- eigenvectors ---
def _euler_flux(U, d, g):
    rho, m, E = U[0], U[1:4], U[4]
    u = m / rho
    p = (g - 1.0) * (E - 0.5 * rho * np.dot(u, u))
    F = np.empty(5, dtype=U.dtype)
    F[0] = m[d]
    F[1:4] = m[d] * u
    F[1 + d] += p
    F[4] = (E + p) * u[d]
    return F


@pytest.mark.parametrize("d", [0, 1, 2])
def test_eigenvectors_diagonalise_jacobian(d):
    """L R = I and L A R = diag(u-c, u, u, u, u+c), A = dF/dU by complex step
    of the Euler flux."""
    g = 1.4
    rng = np.random.default_rng(11 + d)
    for _ in range(3):
        rho = rng.uniform(0.5, 2)
        u = rng.normal(size=3)
        p = rng.uniform(0.5, 2)
        E = p / (g - 1) + 0.5 * rho * np.dot(u, u)
        H = (E + p) / rho
        L, R, c = O.eigvec(g, d, u, H)
        assert np.allclose(L @ R, np.eye(5), atol=1e-12)
        U = np.array([rho, *(rho * u), E])
        A = np.zeros((5, 5))
        hh = 1e-30
        for k in range(5):
            Uc = U.astype(complex)
            Uc[k] += 1j * hh
            A[:, k] = _euler_flux(Uc, d, g).imag / hh
        lam = L @ A @ R
        expect = np.diag([u[d] - c, u[d], u[d], u[d], u[d] + c])
        assert np.allclose(lam, expect, atol=1e-11)
        assert abs(c - np.sqrt(g * p / rho)) < 1e-13


# --------------------------------------------------------------- RK3 ---
def test_rk3_third_order_and_consistency():
    e = [abs(O.rk3_scalar(-1.0, 1.0, 1.0 / n, n) - np.exp(-1.0)) for n in (20, 40, 80)]
    r1, r2 = np.log2(e[0] / e[1]), np.log2(e[1] / e[2])
    assert 2.8 < r1 < 3.2 and 2.8 < r2 < 3.2
    # one step of y' = lambda y reproduces the cubic Taylor polynomial
    z = 0.1
    assert abs(O.rk3_scalar(1.0, 1.0, z, 1) - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


# ------------------------------------------------------------- metric ---
def test_metric_uniform_and_periodic_stretched():
    p = _prob(8, 16, 8)
    ey, eyy = O.metric(p)
    assert np.allclose(ey, 16 / (2 * np.pi), rtol=1e-13) and np.allclose(eyy, 0, atol=1e-9)
    errs = []
    for ny in (16, 32):
        xi = np.arange(ny) * 2 * np.pi / ny
        A = 0.3
        y = xi + A * np.sin(xi)
        p = _prob(4, ny, 4, y=y)
        ey, eyy = O.metric(p)
        h = 2 * np.pi / ny
        yx = 1 + A * np.cos(xi)      # dy/dxi
        yxx = -A * np.sin(xi)
        ey_ex = 1.0 / (yx * h)       # deta/dy with eta = xi/h
        eyy_ex = -(yxx * h * h) / (yx * h) ** 3
        errs.append((np.max(np.abs(ey / ey_ex - 1)), np.max(np.abs(eyy - eyy_ex) / np.max(np.abs(eyy_ex)))))
    assert np.log2(errs[0][0] / errs[1][0]) > 5.5
    assert np.log2(errs[0][1] / errs[1][1]) > 5.5


def test_metric_wall_mirror_interior_order():
    """With walls, nodes at least 3 away from the walls see only true nodes
    and converge at 6th order to the analytic tanh map."""
    out = []
    for ny in (32, 64):
        beta = 1.8
        y = W.tanh_nodes(ny, beta)
        p = O.Problem(4, ny, 4, 1.0, 2.0, 1.0, y=y, wall_y=True)
        ey, _ = O.metric(p)
        xi = -1 + (np.arange(ny) + 0.5) * 2 / ny
        h = 2.0 / ny
        yx = beta / np.cosh(beta * xi) ** 2 / np.tanh(beta)
        j = np.arange(3, ny - 3)
        xs = xi[j]
        sel = np.abs(xs) < 0.5  # same physical region at both resolutions
        out.append(np.max(np.abs(ey[j][sel] * yx[j][sel] * h - 1)))
    assert np.log2(out[0] / out[1]) > 5.5


# ------------------------------------------------- discrete properties ---
@pytest.mark.parametrize("weno", [0, 1, 3, 5, 7])
def test_free_stream_exact(weno):
    """A uniform state has R = 0 exactly, uniform and stretched y, central
    and WENO-forced, viscous."""
    for stretched in (False, True):
        y = None
        if stretched:
            xi = np.arange(12) * 2 * np.pi / 12
            y = xi + 0.3 * np.sin(xi)
        p = _prob(10, 12, 9, y=y, mach=0.4, re=50.0, weno_order=weno, threshold=-1.0)
        one = np.ones((9, 12, 10))
        w = W.conserved(1.2 * one, 0.3 * one, -0.2 * one, 0.1 * one, 1.1 * one, 1.4, 0.4)
        # the inviscid fluxes cancel exactly; the second-derivative stencil of
        # a constant is zero only up to the rounding of its coefficients
        assert np.max(np.abs(O.rhs(p, w, terms=O.CONV))) == 0.0
        assert np.max(np.abs(O.rhs(p, w))) < 1e-13


def test_quiescent_walls_fixed_point():
    y = W.tanh_nodes(16, 1.5)
    p = O.Problem(8, 16, 6, 3.0, 2.0, 2.0, y=y, wall_y=True, t_wall=1.0, mach=1.5, re=300.0,
                  weno_order=5, threshold=-1.0, force=True)
    one = np.ones((6, 16, 8))
    w = W.conserved(one, 0 * one, 0 * one, 0 * one, one, 1.4, 1.5)
    assert np.max(np.abs(O.rhs(p, w, terms=O.CONV))) == 0.0
    assert np.max(np.abs(O.rhs(p, w))) < 1e-12


@pytest.mark.parametrize("weno", [0, 1, 3, 5, 7])
def test_discrete_conservation_periodic(weno):
    """Flux form: sum over a periodic box of every inviscid R is round-off,
    with stretched y weighted by the cell volume 1/eta_y; with constant
    viscosity mass and momentum stay conserved."""
    xi = np.arange(14) * 2 * np.pi / 14
    y = xi + 0.25 * np.sin(xi)
    p = _prob(12, 14, 10, y=y, mach=0.6, re=-1.0, weno_order=weno, threshold=0.3)
    w = W.smooth_periodic(12, 14, 10, seed=5, mach=0.6, amp_u=0.8, amp_s=0.3)
    r, flags = O.rhs(p, w, flags=True)
    if weno:
        frac = np.mean(np.concatenate([f.ravel() for f in flags]))
        assert 0.05 < frac < 0.95  # both branches active
    ey, _ = O.metric(p)
    dv = (1.0 / ey)[None, None, :, None]
    tot = np.sum(r * dv, axis=(1, 2, 3))
    scale = np.sum(np.abs(r) * dv, axis=(1, 2, 3))
    assert np.all(np.abs(tot) < 1e-13 * scale)
    # constant viscosity: mass and momentum
    p2 = _prob(12, 14, 10, mach=0.6, re=20.0, visc_exp=0.0, weno_order=0)
    r2 = O.rhs(p2, w, terms=O.VISC)
    tot2 = np.sum(r2, axis=(1, 2, 3))
    sc2 = np.sum(np.abs(r2), axis=(1, 2, 3))
    assert np.all(np.abs(tot2[1:4]) < 1e-13 * sc2[1:4])


def _d1_periodic(f, axis, h, order=6):
    out = np.zeros_like(f)
    for l, a in enumerate(central_coeffs(order), start=1):
        out += a * (np.roll(f, -l, axis=axis) - np.roll(f, l, axis=axis))
    return out / h


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_kinetic_energy_preservation(order):
    """Inviscid split form: sum(u.R_mom - |u|^2/2 R_rho) equals the pressure
    work sum(p div_h u) exactly (the convective part conserves kinetic
    energy), on random smooth periodic fields, for every central order."""
    n = (14, 12, 10)
    p = _prob(n[0], n[1], n[2], mach=0.5, re=-1.0, weno_order=0, central_order=order)
    w = W.smooth_periodic(*n, seed=21, mach=0.5, amp_u=0.7, amp_s=0.3)
    r = O.rhs(p, w, terms=O.CONV)
    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    R = 1 / (1.4 * 0.25)
    T = (w[4] / rho - 0.5 * (u * u + v * v + ww * ww)) / (R / 0.4)
    pr = rho * R * T
    h = [2 * np.pi / m for m in n]
    lhs = np.sum(u * r[1] + v * r[2] + ww * r[3] - 0.5 * (u * u + v * v + ww * ww) * r[0])
    div = _d1_periodic(u, 2, h[0], order) + _d1_periodic(v, 1, h[1], order) + _d1_periodic(ww, 0, h[2], order)
    rhs_ = np.sum(pr * div)
    scale = np.sum(np.abs(u * r[1])) + np.sum(np.abs(pr * div))
    assert abs(lhs - rhs_) < 1e-13 * scale
    # and the identity is not trivially satisfied
    assert abs(rhs_) > 1e-6 * scale


@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_modified_wavenumber_entropy_wave(axis, order):
    """Density wave at uniform velocity and pressure: R_rho is exactly
    -U eps cos(k x) times the closed-form modified wavenumber."""
    n = 16
    k = 3
    h = 2 * np.pi / n
    x = np.arange(n) * h
    eps, U = 0.1, 0.7
    shape = (n, n, n)
    X = np.meshgrid(x, x, x, indexing="ij")[2 - axis]  # coordinate along `axis` (x is last)
    rho = 1.0 + eps * np.sin(k * X)
    vel = [np.zeros(shape)] * 3
    vel = [np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    vel[axis] = U * np.ones(shape)
    R = 1 / (1.4 * 0.3 ** 2)
    T = 1.0 / rho  # p = R uniform
    w = W.conserved(rho, vel[0], vel[1], vel[2], T, 1.4, 0.3)
    p = _prob(n, n, n, mach=0.3, re=-1.0, central_order=order)
    r = O.rhs(p, w, terms=O.CONV)
    exact = -U * eps * np.cos(k * X) * mod_wavenumber(k, h, order)
    assert np.max(np.abs(r[0] - exact)) < 1e-12
    assert np.max(np.abs(r[1 + axis] - U * exact)) < 1e-12


# ----------------------------------------------------------------- sensor ---
def test_sensor_closed_forms():
    n = 16
    h = 2 * np.pi / n
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    A = 0.8
    one = np.ones_like(X)
    # 1-D compression/expansion: u = -A sin x  -> theta = -A k' cos x, omega = 0
    w = W.conserved(one, -A * np.sin(X), 0 * one, 0 * one, one, 1.4, 0.5)
    s, d = O.sensor(_prob(n, n, n, mach=0.5), w)
    kp = mod_wavenumber(1, h)
    th = -A * kp * np.cos(X)
    assert np.allclose(d, th, atol=1e-13)
    assert np.allclose(s, np.maximum(-th / np.sqrt(th * th + 1.0), 0.0), atol=1e-14)
    # solenoidal Taylor-Green velocity: theta = 0 to round-off, sensor 0
    c = W.taylor_green(n)
    s2, d2 = O.sensor(_prob(n, n, n, mach=c.mach), c.w0)
    assert np.max(np.abs(d2)) < 1e-12 and np.max(s2) < 1e-12


# ----------------------------------------------------- manufactured RHS ---
def _ns_rhs_exact(fields, mach, re, pr, gamma, visc_exp):
    """Analytic compressible Navier-Stokes RHS (divergence form) of the
    closed-form fields (rho, u, v, w, T) of x, y, z."""
    x, y, z = sp.symbols("x y z")
    rho, u, v, w, T = fields
    R = 1 / (gamma * mach ** 2)
    cp = gamma * R / (gamma - 1)
    p = rho * R * T
    H = cp * T + (u * u + v * v + w * w) / 2
    U = [u, v, w]
    X = [x, y, z]
    mu = T ** visc_exp / re
    kc = mu * cp / pr
    th = sum(sp.diff(U[a], X[a]) for a in range(3))
    tau = [[mu * (sp.diff(U[a], X[b]) + sp.diff(U[b], X[a]) - (sp.Rational(2, 3) * th if a == b else 0))
            for b in range(3)] for a in range(3)]
    out = [-sum(sp.diff(rho * U[j], X[j]) for j in range(3))]
    for i in range(3):
        out.append(-sum(sp.diff(rho * U[i] * U[j] + (p if i == j else 0), X[j]) for j in range(3))
                   + sum(sp.diff(tau[i][j], X[j]) for j in range(3)))
    out.append(-sum(sp.diff(rho * U[j] * H, X[j]) for j in range(3))
               + sum(sp.diff(sum(U[i] * tau[i][j] for i in range(3)) + kc * sp.diff(T, X[j]), X[j])
                     for j in range(3)))
    f = [sp.lambdify((x, y, z), e, "numpy") for e in fields]
    r = [sp.lambdify((x, y, z), e, "numpy") for e in out]
    return f, r


def _mms_exact(mach, re, pr, gamma, visc_exp):
    x, y, z = sp.symbols("x y z")
    rho = 1 + sp.Rational(1, 5) * sp.sin(x + sp.Rational(3, 10)) * sp.cos(y) + sp.sin(z) / 10
    u = sp.sin(y + z) / 2 + sp.cos(x) / 5
    v = sp.Rational(2, 5) * sp.cos(x + z) - sp.sin(y) / 10
    w = sp.Rational(3, 10) * sp.sin(x - y) + sp.cos(z) / 5
    T = 1 + sp.cos(x) * sp.sin(y + z) / 10
    return _ns_rhs_exact((rho, u, v, w, T), mach, re, pr, gamma, visc_exp)


@pytest.fixture(scope="module")
def mms():
    return _mms_exact(0.5, 100.0, 0.72, 1.4, 0.76)


@pytest.mark.parametrize("stretched,order", [(False, 6), (True, 6), (False, 2), (False, 4), (False, 8),
                                             (True, 8)])
def test_design_order_manufactured(mms, stretched, order):
    """R_h(w*) - R(w*) falls as h^order for convective (split form) plus
    viscous (Laplacian form) terms of the same order, uniform and stretched
    y (the metric uses the higher of the two orders)."""
    fields, rhs = mms
    errs = []
    # 8th order needs finer grids to leave the pre-asymptotic range
    for n in ((24, 48) if order == 8 else (16, 32)):
        xi = np.arange(n) * 2 * np.pi / n
        yv = xi + 0.3 * np.sin(xi) if stretched else xi
        Z, Y, X = np.meshgrid(xi, yv, xi, indexing="ij")
        vals = [f(X, Y, Z) * np.ones_like(X) for f in fields]
        w = W.conserved(*vals, 1.4, 0.5)
        p = _prob(n, n, n, y=yv if stretched else None, mach=0.5, re=100.0, prandtl=0.72,
                  visc_exp=0.76, weno_order=0, central_order=order, visc_order=order)
        r = O.rhs(p, w)
        ex = np.stack([g(X, Y, Z) * np.ones_like(X) for g in rhs])
        errs.append(np.max(np.abs(r - ex), axis=(1, 2, 3)) / np.max(np.abs(ex), axis=(1, 2, 3)))
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > order - 0.6), rates


@pytest.mark.parametrize("order,min_rate", [(3, 2.0), (5, 4.0), (7, 5.5)])
def test_weno_forced_order_entropy_wave(order, min_rate):
    """WENO everywhere on a smooth entropy wave: the mass RHS converges to
    -U drho/dx at (nearly) the design order."""
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        X = x[None, None, :] * np.ones((1, 1, n))
        rho = 1.0 + 0.2 * np.sin(X)
        one = np.ones_like(X)
        w = W.conserved(rho, 0.6 * one, 0 * one, 0 * one, 1.0 / rho, 1.4, 0.5)
        p = O.Problem(n, 1, 1, 2 * np.pi, 1.0, 1.0, mach=0.5, re=-1.0, weno_order=order, threshold=-1.0)
        r = O.rhs(p, w, terms=O.CONV)
        ex = -0.6 * 0.2 * np.cos(X)
        errs.append(np.mean(np.abs(r[0] - ex)))
    assert np.log2(errs[0] / errs[1]) > min_rate


# ----------------------------------------------------------- wall / forcing ---
def test_channel_reflection_symmetry():
    """A state even in y (rho, T, u, w) with odd v on the symmetric tanh grid
    gives an RHS with the same symmetry: both walls use consistent
    mirror maps."""
    ny = 16
    y = W.tanh_nodes(ny, 1.6)
    nx, nz = 8, 6
    rng = np.random.default_rng(2)
    x = np.arange(nx) * 2 * np.pi / nx
    z = np.arange(nz) * 2 * np.pi / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ph = rng.uniform(0, 6, 4)
    rho = 1 + 0.1 * np.cos(X + ph[0]) * (1 - Y ** 2)
    T = 1 + 0.2 * (1 - Y ** 4) + 0.05 * np.sin(Z + ph[1])
    u = 1.5 * (1 - Y ** 2) * (1 + 0.1 * np.sin(X + Z))
    v = 0.1 * Y * (1 - Y ** 2) * np.cos(X + ph[2])
    ww = 0.1 * (1 - Y ** 2) * np.sin(Z + ph[3])
    w = W.conserved(rho, u, v, ww, T, 1.4, 1.5)
    p = O.Problem(nx, ny, nz, 2 * np.pi, 2.0, 2 * np.pi, y=y, wall_y=True, mach=1.5, re=300.0,
                  weno_order=5, threshold=0.05, force=True)
    r = O.rhs(p, w)
    par = np.array([1, 1, -1, 1, 1])
    flipped = r[:, :, ::-1, :] * par[:, None, None, None]
    scale = np.max(np.abs(r), axis=(1, 2, 3))[:, None, None, None]
    assert np.max(np.abs(flipped - r) / scale) < 1e-12


def test_forcing_keeps_bulk_momentum():
    c = W.channel(16, 16, 8, seed=99)
    p = O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, y=c.y, wall_y=True, mach=c.mach, re=c.re,
                  force=True, weno_order=5)
    ey, _ = O.metric(p)
    dv = (1.0 / ey)[None, :, None]
    b0 = np.sum(c.w0[1] * dv)
    w, _, _ = O.step(p, c.w0, 3, dt_fixed=2e-3)
    assert abs(np.sum(w[1] * dv) - b0) < 1e-13 * abs(b0)
    r = O.rhs(p, w)
    assert abs(np.sum(r[1] * dv)) < 1e-12 * np.sum(np.abs(r[1]) * dv)


def test_dt_closed_form_uniform():
    p = _prob(8, 8, 8, mach=0.5, re=200.0, prandtl=0.7)
    one = np.ones((8, 8, 8))
    w = W.conserved(1.3 * one, 0.4 * one, -0.3 * one, 0.2 * one, 1.2 * one, 1.4, 0.5)
    R = 1 / (1.4 * 0.25)
    c = np.sqrt(1.4 * R * 1.2)
    h = 2 * np.pi / 8
    conv = (0.4 + c + 0.3 + c + 0.2 + c) / h
    visc = 1.4 * (1.2 ** 0.76 / 200.0) / (0.7 * 1.3) * 3 / h ** 2
    assert abs(O.dt(p, w, 0.8) - 0.8 / (conv + visc)) < 1e-14


# --------------------------------------------------------- exact solutions ---
def _golden(name):
    """name -> (value, tolerance) from a fixture under tests/golden/."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


def test_riemann_solver_textbook_values():
    """Star state of Sod's problem as tabulated by Toro (Table 4.3;
    tests/golden/sod_star_state.txt)."""
    g = _golden("sod_star_state.txt")
    ps, us = ER.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - g["p_star"][0]) < g["p_star"][1]
    assert abs(us - g["u_star"][0]) < g["u_star"][1]


def test_sod_exact_solution():
    """Double Sod problem, WENO5 everywhere, t = 0.2: density close to the
    exact solution in L1 and first-order convergence."""
    errs = []
    for n in (200, 400):
        w0, x, mach = W.double_sod(n)
        p = O.Problem(n, 1, 1, 2.0, 1.0, 1.0, mach=mach, re=-1.0, weno_order=5, threshold=-1.0)
        dtv = 0.2 / (n // 2)
        w, _, _ = O.step(p, w0, n // 2, dt_fixed=dtv)
        rho = w[0, 0, 0]
        # right-moving Sod at x = 1.5 and its mirror at x = 0.5
        ex = np.where(x >= 1.0,
                      ER.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 1.5) / 0.2)[0],
                      ER.sample((0.125, 0.0, 0.1), (1.0, 0.0, 1.0), (x - 0.5) / 0.2)[0])
        errs.append(np.mean(np.abs(rho - ex)) * 2.0)
        assert np.all(np.isfinite(w))
        # mirror symmetry about x = 1
        assert np.max(np.abs(rho - rho[::-1])) < 1e-10
    assert errs[1] < 0.012
    assert errs[0] / errs[1] > 1.5


def test_isentropic_vortex_translation():
    """Shu's vortex is carried unchanged by the uniform stream: after one
    period the density matches the initial field, converging with h."""
    errs = []
    for n in (24, 48):
        w0, mach = W.isentropic_vortex(n)
        p = O.Problem(n, n, 1, 10.0, 10.0, 1.0, mach=mach, re=-1.0, weno_order=0)
        nsteps = 4 * n
        w, _, _ = O.step(p, w0, nsteps, dt_fixed=10.0 / nsteps)
        errs.append(np.max(np.abs(w[0] - w0[0])))
    assert errs[1] < 2e-3
    assert np.log2(errs[0] / errs[1]) > 2.8


def test_design_order_manufactured_walls():
    """Isothermal no-slip walls: fields whose mirror continuation is analytic
    (velocity and T - T_w odd about each wall, pressure even) make the whole
    RHS, wall rows included, converge at 6th order.  This pins the ghost
    rules of velocity, temperature, density and the stored divergence."""
    x, y, z = sp.symbols("x y z")
    mach, tw = 0.8, 1.0
    R = 1 / (1.4 * mach ** 2)
    cy, sy = sp.cos(sp.pi * y / 2), sp.sin(sp.pi * y)
    u = (sp.Rational(3, 2) + sp.sin(x + z) / 5) * cy
    v = sp.Rational(3, 10) * sy * sp.cos(x)
    w = sp.Rational(2, 5) * cy * sp.sin(z)
    T = tw + sp.Rational(3, 10) * cy * (1 + sp.cos(x) / 10)
    p = R * (1 + sp.cos(sp.pi * y) * sp.cos(z) / 10)
    rho = p / (R * T)
    fields, rhs = _ns_rhs_exact((rho, u, v, w, T), mach, 50.0, 0.72, 1.4, 0.76)
    errs = []
    for ny in (16, 32):
        nx = nz = ny // 2
        xs = np.arange(nx) * 2 * np.pi / nx
        zs = np.arange(nz) * 2 * np.pi / nz
        ys = -1.0 + (np.arange(ny) + 0.5) * 2.0 / ny
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        vals = [f(X, Y, Z) * np.ones_like(X) for f in fields]
        wv = W.conserved(*vals, 1.4, mach)
        pr = O.Problem(nx, ny, nz, 2 * np.pi, 2.0, 2 * np.pi, wall_y=True, t_wall=tw, mach=mach,
                       re=50.0, weno_order=0)
        r = O.rhs(pr, wv)
        ex = np.stack([g(X, Y, Z) * np.ones_like(X) for g in rhs])
        errs.append(np.max(np.abs(r - ex), axis=(1, 2, 3)) / np.max(np.abs(ex), axis=(1, 2, 3)))
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > 5.0), rates


def test_forcing_is_body_force_with_its_power():
    """The forcing adds a uniform x force f to the x momentum and its power
    f u to the energy, nothing else, with f closing the volume balance."""
    c = W.channel(12, 16, 8, seed=5)
    p = O.Problem(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz, y=c.y, wall_y=True, mach=c.mach, re=c.re,
                  force=True, weno_order=5)
    full = O.rhs(p, c.w0)
    base = O.rhs(p, c.w0, terms=O.CONV | O.VISC)
    d = full - base
    f = d[1].ravel()[0]
    assert abs(f) > 0
    assert np.allclose(d[1], f, rtol=1e-12, atol=0)
    assert np.max(np.abs(d[[0, 2, 3]])) == 0.0
    assert np.allclose(d[4], f * c.w0[1] / c.w0[0], rtol=1e-12, atol=1e-15)


# --------------------------------------------- characteristic WENO flux ---
def _linear_upwind_coeffs(order):
    """Coefficients c_m, m = -(r-1) .. r-1, of the linear (optimal-weight)
    reconstruction at x_{i+1/2} from the left, derived symbolically here."""
    fs, qs, _, d = _jiang_shu_reference(order)
    lin = sp.expand(sum(d[k] * qs[k] for k in range(len(qs))))
    return np.array([float(lin.coeff(f)) for f in fs])


def _upwind_symbol_rhs(order, speed, eps, k, h, x):
    """-(speed/h) times the flux difference of the linear upwind
    reconstruction of eps sin(k x), taken from the side the wave comes from:
    F_{i+1/2} = speed sum_m c_m f_{i+m} (speed > 0) or speed sum_m c_m
    f_{i+1-m} (speed < 0)."""
    c = _linear_upwind_coeffs(order)
    r = (order + 1) // 2
    m = np.arange(-(r - 1), r)
    shift = m if speed > 0 else 1 - m
    S = np.sum(c * np.exp(1j * k * shift * h))
    return -(speed * eps / h) * np.imag(np.exp(1j * k * x) * S * (1.0 - np.exp(-1j * k * h)))


def _central_symbol_rhs(order, speed, eps, k, h, x):
    """The same with the non-dissipative central reconstruction of the same
    stencil width (the mean of the left and right linear reconstructions)."""
    return 0.5 * (_upwind_symbol_rhs(order, speed, eps, k, h, x) + _upwind_symbol_rhs(order, -speed, eps, k, h, x)
                  * -1.0)


@pytest.mark.parametrize("order", [1, 3, 5, 7])
@pytest.mark.parametrize("U", [0.6, -0.45])
def test_weno_entropy_wave_linear_upwind_symbol(order, U):
    """Small-amplitude entropy wave (velocity U and pressure uniform), WENO at
    every interface, inviscid.  With amplitude 1e-8 the nonlinear weights equal
    the linear ones to ~1e-9, and the characteristic Lax-Friedrichs flux of
    the mass equation is exactly U times the linear upwind reconstruction of
    rho from the side the flow comes from -- but only if the entropy field is
    split with its own dissipation max|u_n| = |U| (one alpha per
    characteristic field).  With one alpha = max(|u_n| + c) for every field the
    entropy wave would get the extra dissipation (c/2)(upwind - downwind),
    some 1e-3 of R_rho here.  R_rho must equal the closed-form symbol of the
    upwind scheme to 1e-6."""
    n, k, eps, mach = 32, 5, 1e-8, 0.5
    h = 2 * np.pi / n
    x = np.arange(n) * h
    X = x[None, None, :] * np.ones((1, 1, n))
    rho = 1.0 + eps * np.sin(k * X)
    one = np.ones_like(X)
    w = W.conserved(rho, U * one, 0 * one, 0 * one, 1.0 / rho, 1.4, mach)  # p = rho R T uniform
    p = O.Problem(n, 1, 1, 2 * np.pi, 1.0, 1.0, mach=mach, re=-1.0, weno_order=order, threshold=-1.0)
    r = O.rhs(p, w, terms=O.CONV)
    exact = _upwind_symbol_rhs(order, U, eps, k, h, x)
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(r[0, 0, 0] - exact)) < 1e-6 * scale
    # the momentum row follows the mass flux (u uniform); its flux carries
    # the pressure, ~300 times R_rho here, hence the rounding allowance
    assert np.max(np.abs(r[1, 0, 0] - U * exact)) < 1e-5 * abs(U) * scale
    # the test resolves the dissipation: the central symbol of the same width is far off
    if order > 1:
        central = _central_symbol_rhs(order, U, eps, k, h, x)
        assert np.max(np.abs(central - exact)) > 1e-4 * scale


@pytest.mark.parametrize("order", [3, 5, 7])
@pytest.mark.parametrize("sign", [1, -1])
def test_weno_acoustic_wave_linear_upwind_symbol(order, sign):
    """Small-amplitude acoustic wave carried by the u + sign*c field alone
    (rho' = eps s, u' = sign c eps s, p' = c^2 eps s, s = sin kx) on a flow
    at U = 0.3, c = 2, WENO everywhere: every conserved field's RHS is the
    linear upwind symbol at the speed U + sign*c, taken from that speed's
    upwind side, up to O(eps) relative.  Pins the eigenvectors (no leak into
    the other fields), the side each field is upwinded from and the
    acoustic fields' dissipation."""
    n, k, eps, mach, U, g = 32, 5, 1e-8, 0.5, 0.3, 1.4
    c0 = 1.0 / mach  # T = 1: c^2 = gamma R T = 1/M^2
    h = 2 * np.pi / n
    x = np.arange(n) * h
    X = x[None, None, :] * np.ones((1, 1, n))
    s = np.sin(k * X)
    Rg = 1.0 / (g * mach * mach)
    rho = 1.0 + eps * s
    u = U + sign * c0 * eps * s
    pr = Rg + c0 * c0 * eps * s
    one = np.ones_like(X)
    w = W.conserved(rho, u, 0 * one, 0 * one, pr / (rho * Rg), g, mach)
    p = O.Problem(n, 1, 1, 2 * np.pi, 1.0, 1.0, mach=mach, re=-1.0, weno_order=order, threshold=-1.0)
    r = O.rhs(p, w, terms=O.CONV)
    lam = U + sign * c0
    exact = _upwind_symbol_rhs(order, lam, eps, k, h, x)
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(r[0, 0, 0] - exact)) < 1e-6 * scale
    # momentum: d(rho u)' = u0 rho' + rho0 u' = (U + sign c) eps s
    assert np.max(np.abs(r[1, 0, 0] - (U + sign * c0) * exact)) < 1e-6 * abs(U + sign * c0) * scale
    assert np.max(np.abs(r[2:4])) < 1e-6 * scale


def test_roe_average_property_calorically_perfect():
    """Roe's property of the sqrt(rho)-weighted state of the WENO flux: with
    A~ = R diag(u_n - c, u_n, u_n, u_n, u_n + c) L at that state,
    A~ (w_b - w_a) = F(w_b) - F(w_a) exactly, for any two states of a
    calorically perfect gas (Roe 1981).  An arithmetic mean of H or u, or a
    sound speed not from (gamma-1)(H - |u|^2/2), breaks it."""
    g, mach = 1.4, 0.5
    Rg = 1.0 / (g * mach * mach)
    cv = Rg / (g - 1.0)
    p = O.Problem(4, 4, 4, 1.0, 1.0, 1.0, mach=mach, gamma=g)
    rng = np.random.default_rng(17)
    for d in range(3):
        for _ in range(20):
            sa = np.array([rng.uniform(0.2, 3.0), *rng.normal(size=3), rng.uniform(0.3, 3.0)])
            sb = np.array([rng.uniform(0.2, 3.0), *rng.normal(size=3), rng.uniform(0.3, 3.0)])
            roe = O.roe_state(p, sa, sb)
            L, R, c = O.eigvec(g, d, roe[:3], roe[3])
            assert abs(roe[5] - c) <= 1e-14 * c
            lam = np.diag([roe[d] - c, roe[d], roe[d], roe[d], roe[d] + c])
            A = R @ lam @ L

            def cons(st):
                rho, vel, T = st[0], st[1:4], st[4]
                return np.array([rho, *(rho * vel), rho * (cv * T + 0.5 * np.dot(vel, vel))])

            wa, wb = cons(sa), cons(sb)
            dF = _euler_flux(wb, d, g) - _euler_flux(wa, d, g)
            scale = np.max(np.abs(_euler_flux(wb, d, g))) + np.max(np.abs(_euler_flux(wa, d, g)))
            assert np.max(np.abs(A @ (wb - wa) - dF)) < 1e-12 * scale


def test_weno7_indicator_evaluation_form():
    """The WENO7 smoothness indicators are one quadratic form of the stencil
    values (240 x the Jiang-Shu integral).  The oracle evaluates it as a
    weighted sum of squares of undivided differences; the alternative is the
    expanded form sum_ij C_ij f_i f_j.  Against the exact rational value of
    the integral definition (fractions.Fraction), on stencils with a common
    offset much larger than their variation -- characteristic fluxes near a
    mean state -- the sum of squares stays within a few 1e-7 relative while
    the expanded form loses every digit to cancellation; on unit-scale data
    both are at rounding level.  This, not agreement with another
    implementation, is why the oracle uses that form."""
    from fractions import Fraction

    fs, _, bs, _ = _jiang_shu_reference(7)
    polys = [sp.Poly(sp.expand(240 * b), *fs) for b in bs]
    terms = [[(tuple(mon), Fraction(int(sp.fraction(cf)[0]), int(sp.fraction(cf)[1])))
              for mon, cf in P.terms()] for P in polys]

    def exact(f):
        fr = [Fraction(float(v)) for v in f]
        out = []
        for tt in terms:
            acc = Fraction(0)
            for mon, cf in tt:
                t = cf
                for i, e in enumerate(mon):
                    if e:
                        t *= fr[i] ** e
                acc += t
            out.append(acc)
        return out

    def expanded(f):
        out = []
        for tt in terms:
            acc = 0.0
            for mon, cf in tt:
                t = float(cf)
                for i, e in enumerate(mon):
                    for _ in range(e):
                        t *= float(f[i])
                acc += t
            out.append(acc)
        return out

    rng = np.random.default_rng(29)
    err_sos = {"offset": 0.0, "unit": 0.0}
    err_exp = {"offset": 0.0, "unit": 0.0}
    for trial in range(120):
        kind = "offset" if trial % 2 == 0 else "unit"
        if kind == "offset":
            f = rng.uniform(-1e3, 1e3) + rng.normal(size=7) * 10.0 ** rng.uniform(-5, -1)
        else:
            f = rng.normal(size=7)
        ex = exact(f)
        _, b = O.weno_parts(7, f)
        be = expanded(f)
        for kk in range(4):
            ref = float(ex[kk])
            err_sos[kind] = max(err_sos[kind], abs(b[kk] - ref) / ref)
            err_exp[kind] = max(err_exp[kind], abs(be[kk] - ref) / ref)
    assert err_sos["unit"] < 1e-13 and err_exp["unit"] < 1e-12
    assert err_sos["offset"] < 1e-6
    assert err_exp["offset"] > 1e3 * err_sos["offset"]


# --------------------------------------------------------------- KEEP-n ---
def _entropy_vars(w, gamma=1.4):
    """Entropy variables of U = -rho s/(gamma-1), s = ln(p rho^-gamma)."""
    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    q2 = u * u + v * v + ww * ww
    p = (gamma - 1.0) * (w[4] - 0.5 * rho * q2)
    s = np.log(p) - gamma * np.log(rho)
    b = rho / p
    return np.stack([(gamma - s) / (gamma - 1.0) - 0.5 * b * q2, b * u, b * v, b * ww, -b])


def _entropy_production(keep, order, stretched=False, seed=31):
    n = (14, 12, 10)
    xi = np.arange(n[1]) * 2 * np.pi / n[1]
    y = xi + 0.25 * np.sin(xi) if stretched else None
    p = _prob(n[0], n[1], n[2], y=y, mach=0.5, re=-1.0, weno_order=0, central_order=order, keep=keep)
    w = W.smooth_periodic(*n, seed=seed, mach=0.5, amp_u=0.6, amp_s=0.3)
    r = O.rhs(p, w, terms=O.CONV)
    ey, _ = O.metric(p)
    dv = (1.0 / ey)[None, :, None]
    prod = np.sum(_entropy_vars(w) * r, axis=0)
    return abs(np.sum(prod * dv)) / np.sum(np.abs(prod) * dv)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("stretched", [False, True])
def test_keep_conserves_entropy(order, stretched):
    """KEEP with exact logarithmic means: the inviscid central RHS conserves
    the entropy -rho s/(gamma-1) exactly (sum of v . R dV over a periodic
    box is round-off, v the entropy variables, dV = 1/eta_y), by Tadmor's
    condition of the two-point flux and the antisymmetric flux-
    differencing form; the split form of the default scheme does not."""
    assert _entropy_production(-1, order, stretched) < 1e-12
    assert _entropy_production(0, order, stretched) > 1e-5


def test_keep_n_entropy_error_falls_with_n():
    """KEEP-n: logarithmic means from n terms of their series; the entropy
    production falls with the number of terms (error of order z^2n)."""
    e = {n: _entropy_production(n, 6) for n in (1, 2, 5, 6)}
    # (the net production sums signed per-pair errors, so single steps of n
    # can cancel; the trend over several terms cannot)
    assert e[1] > 10 * e[2] > 1000 * e[5]
    assert e[6] < 1e-11


@pytest.mark.parametrize("keep", [-1, 2])
def test_keep_preserves_kinetic_energy_and_pressure_equilibrium(keep):
    """KEEP's momentum flux (mass flux times the mean velocity plus the mean
    pressure) gives the split form's kinetic-energy identity
    sum(u.R_mom - |u|^2/2 R_rho) = sum(p div_h u); with uniform velocity and
    pressure and a varying density, the pressure stays uniform (dp/dt = 0),
    which the split form with the total enthalpy does not give."""
    n = (14, 12, 10)
    p = _prob(n[0], n[1], n[2], mach=0.5, re=-1.0, weno_order=0, keep=keep)
    w = W.smooth_periodic(*n, seed=21, mach=0.5, amp_u=0.7, amp_s=0.3)
    r = O.rhs(p, w, terms=O.CONV)
    rho = w[0]
    u, v, ww = w[1] / rho, w[2] / rho, w[3] / rho
    Rg = 1 / (1.4 * 0.25)
    T = (w[4] / rho - 0.5 * (u * u + v * v + ww * ww)) / (Rg / 0.4)
    pr = rho * Rg * T
    h = [2 * np.pi / m for m in n]
    lhs = np.sum(u * r[1] + v * r[2] + ww * r[3] - 0.5 * (u * u + v * v + ww * ww) * r[0])
    div = _d1_periodic(u, 2, h[0]) + _d1_periodic(v, 1, h[1]) + _d1_periodic(ww, 0, h[2])
    rhs_ = np.sum(pr * div)
    scale = np.sum(np.abs(u * r[1])) + np.sum(np.abs(pr * div))
    assert abs(lhs - rhs_) < 1e-13 * scale
    # pressure equilibrium
    shape = (n[2], n[1], n[0])
    rng = np.random.default_rng(4)
    x = np.arange(n[0]) * h[0]
    rho2 = 1.0 + 0.3 * np.sin(x)[None, None, :] * np.ones(shape) + 0.05 * rng.uniform(-1, 1, shape)
    U0 = [0.4 * np.ones(shape), -0.3 * np.ones(shape), 0.2 * np.ones(shape)]
    w2 = W.conserved(rho2, *U0, 1.0 / rho2, 1.4, 0.5)  # p = R uniform
    out = {}
    for k in (keep, 0):
        r2 = O.rhs(_prob(n[0], n[1], n[2], mach=0.5, re=-1.0, weno_order=0, keep=k), w2, terms=O.CONV)
        # dp/dt = (gamma-1) (R_E - u . R_mom + |u|^2/2 R_rho) at uniform u
        uu = [f[0, 0, 0] for f in U0]
        dp = 0.4 * (r2[4] - uu[0] * r2[1] - uu[1] * r2[2] - uu[2] * r2[3] + 0.5 * sum(c * c for c in uu) * r2[0])
        out[k] = np.max(np.abs(dp)) / np.max(np.abs(r2[4]))
    # (dp/dt is a difference of terms each of the size of R_E: rounding
    # level is ~1e-12 of it)
    assert out[keep] < 1e-11
    assert out[0] > 1e-6


def test_keep_design_order_and_conservation(mms):
    """KEEP is a consistent central scheme of the chosen order: R_h(w*) -
    R(w*) falls as h^6 with the 6th-order coefficients (viscous terms
    included); its flux form conserves mass, momentum and energy to
    round-off on a stretched periodic box, with and without WENO."""
    fields, rhs = mms
    errs = []
    for n in (16, 32):
        xi = np.arange(n) * 2 * np.pi / n
        Z, Y, X = np.meshgrid(xi, xi, xi, indexing="ij")
        vals = [f(X, Y, Z) * np.ones_like(X) for f in fields]
        w = W.conserved(*vals, 1.4, 0.5)
        p = _prob(n, n, n, mach=0.5, re=100.0, prandtl=0.72, visc_exp=0.76, weno_order=0, keep=-1)
        r = O.rhs(p, w)
        ex = np.stack([g(X, Y, Z) * np.ones_like(X) for g in rhs])
        errs.append(np.max(np.abs(r - ex), axis=(1, 2, 3)) / np.max(np.abs(ex), axis=(1, 2, 3)))
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > 5.4), rates
    xi = np.arange(14) * 2 * np.pi / 14
    y = xi + 0.25 * np.sin(xi)
    w = W.smooth_periodic(12, 14, 10, seed=5, mach=0.6, amp_u=0.8, amp_s=0.3)
    for weno in (0, 5):
        p = _prob(12, 14, 10, y=y, mach=0.6, re=-1.0, weno_order=weno, threshold=0.3, keep=-1)
        r = O.rhs(p, w)
        ey, _ = O.metric(p)
        dv = (1.0 / ey)[None, None, :, None]
        tot = np.sum(r * dv, axis=(1, 2, 3))
        scale = np.sum(np.abs(r) * dv, axis=(1, 2, 3))
        assert np.all(np.abs(tot) < 1e-13 * scale)
