"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

Written from the published method (E. F. Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", Ch. 4): Newton iteration on the pressure function f_L(p) + f_R(p) + (u_R - u_L) = 0
with the shock / rarefaction branches of f_K, then sampling the self-similar solution at
S = x / t.  Used only as an independent pin of the oracle's hydro scheme.
"""
from __future__ import annotations

import math


def _fk(p, rk, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        pr = p / pk
        f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rk * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(WL, WR, g):
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        pn = max(1e-12, p - (fl + fr + ur - ul) / (dfl + dfr))
        if abs(pn - p) / (0.5 * (pn + p)) < 1e-14:
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(WL, WR, g, S):
    """(rho, u, p) of the exact solution at x/t = S."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(WL, WR, g)
    gm = (g - 1.0) / (g + 1.0)
    if S <= us:  # left of contact
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if S <= sl:
                return rl, ul, pl
            return rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
        shl = ul - cl
        csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        stl = us - csl
        if S <= shl:
            return rl, ul, pl
        if S >= stl:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - S))
        u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + S)
        r = rl * (c / cl) ** (2.0 / (g - 1.0))
        return r, u, pl * (c / cl) ** (2.0 * g / (g - 1.0))
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if S >= sr:
            return rr, ur, pr
        return rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
    shr = ur + cr
    csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    str_ = us + csr
    if S >= shr:
        return rr, ur, pr
    if S <= str_:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - S))
    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + S)
    r = rr * (c / cr) ** (2.0 / (g - 1.0))
    return r, u, pr * (c / cr) ** (2.0 * g / (g - 1.0))


def godunov_flux(WL, WR, g):
    """Exact (Godunov) mass, momentum and energy flux at x/t = 0."""
    r, u, p = sample(WL, WR, g, 0.0)
    E = p / (g - 1.0) + 0.5 * r * u * u
    return r * u, r * u * u + p, u * (E + p)
