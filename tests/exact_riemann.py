"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas: the pressure in the star region from Newton iteration on the
pressure function, then sampling of the self-similar solution (the method of
Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4).
Used to pin the oracle's shock-capturing path against a known solution."""
from __future__ import annotations

import numpy as np


def _f(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    r = p / pk
    f = 2.0 * ck / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _f(p, rl, pl, cl, g)
        fr, dfr = _f(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-10, p - dp)
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g=1.4):
    """(rho, u, p) at the similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    out = np.zeros((3, len(xi)))
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                    out[:, n] = (rs, us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                shl, stl = ul - cl, us - csl
                if s <= shl:
                    out[:, n] = (rl, ul, pl)
                elif s >= stl:
                    out[:, n] = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rho = rl * (c / cl) ** (2.0 / (g - 1))
                    out[:, n] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of contact
            if ps > pr:  # right shock
                sr = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                    out[:, n] = (rs, us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                shr, str_ = ur + cr, us + csr
                if s >= shr:
                    out[:, n] = (rr, ur, pr)
                elif s <= str_:
                    out[:, n] = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rho = rr * (c / cr) ** (2.0 / (g - 1))
                    out[:, n] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
