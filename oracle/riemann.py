"""Exact solution of the 1D Riemann problem of the Euler equations -- test
infrastructure (pins the oracle's Euler scheme, Sec. 3.5, against a closed
form).

Method: E. F. Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", 3rd ed. (2009), Ch. 4: the star pressure p* is the root of
f(p) = f_L(p) + f_R(p) + (u_R - u_L), with f_K the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution is then sampled along x/t.  Written from the equations, in FP64.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, ck, gam):
    if p > pk:
        A = 2.0 / ((gam + 1.0) * rho)
        B = (gam - 1.0) / (gam + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    r = p / pk
    f = 2.0 * ck / (gam - 1.0) * (r ** ((gam - 1.0) / (2.0 * gam)) - 1.0)
    df = 1.0 / (rho * ck) * r ** (-(gam + 1.0) / (2.0 * gam))
    return f, df


def star_state(left, right, gam=1.4, tol=1e-15, maxit=200):
    """(p*, u*) for primitive states left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gam * pl / rl)
    cr = math.sqrt(gam * pr / rr)
    if 2.0 * (cl + cr) / (gam - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    p = max(tol, 0.5 * (pl + pr))       # arithmetic-mean start (Toro Sec. 4.3.2)
    for _ in range(maxit):
        fl, dfl = _f_and_df(p, rl, pl, cl, gam)
        fr, dfr = _f_and_df(p, rr, pr, cr, gam)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, gam)
    fr, _ = _f_and_df(p, rr, pr, cr, gam)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, s, gam=1.4):
    """Primitive state (rho, u, p) at similarity coordinate s = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gam)
    g1 = (gam - 1.0) / (gam + 1.0)
    if s <= us:                                   # left of the contact
        cl = math.sqrt(gam * pl / rl)
        if ps > pl:                               # left shock
            sl = ul - cl * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / pl + (gam - 1.0) / (2.0 * gam))
            if s <= sl:
                return rl, ul, pl
            return rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps
        shl = ul - cl                             # left rarefaction head
        csl = cl * (ps / pl) ** ((gam - 1.0) / (2.0 * gam))
        stl = us - csl
        if s <= shl:
            return rl, ul, pl
        if s >= stl:
            return rl * (ps / pl) ** (1.0 / gam), us, ps
        u = 2.0 / (gam + 1.0) * (cl + (gam - 1.0) / 2.0 * ul + s)
        c = 2.0 / (gam + 1.0) * (cl + (gam - 1.0) / 2.0 * (ul - s))
        rho = rl * (c / cl) ** (2.0 / (gam - 1.0))
        return rho, u, pl * (c / cl) ** (2.0 * gam / (gam - 1.0))
    cr = math.sqrt(gam * pr / rr)                 # right of the contact
    if ps > pr:                                   # right shock
        sr = ur + cr * math.sqrt((gam + 1.0) / (2.0 * gam) * ps / pr + (gam - 1.0) / (2.0 * gam))
        if s >= sr:
            return rr, ur, pr
        return rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps
    shr = ur + cr
    csr = cr * (ps / pr) ** ((gam - 1.0) / (2.0 * gam))
    str_ = us + csr
    if s >= shr:
        return rr, ur, pr
    if s <= str_:
        return rr * (ps / pr) ** (1.0 / gam), us, ps
    u = 2.0 / (gam + 1.0) * (-cr + (gam - 1.0) / 2.0 * ur + s)
    c = 2.0 / (gam + 1.0) * (cr - (gam - 1.0) / 2.0 * (ur - s))
    rho = rr * (c / cr) ** (2.0 / (gam - 1.0))
    return rho, u, pr * (c / cr) ** (2.0 * gam / (gam - 1.0))


def density_profile(left, right, x, x0, t, gam=1.4):
    """Exact density at points x after time t."""
    return np.array([sample(left, right, (xi - x0) / t, gam)[0] for xi in np.ravel(x)]).reshape(np.shape(x))


def cell_average_density(left, right, xlo, dx, x0, t, gam=1.4, nsub=16):
    """Exact cell averages of density over [xlo, xlo+dx] (midpoint rule on nsub sub-cells)."""
    xs = xlo[..., None] + (np.arange(nsub) + 0.5) / nsub * dx
    return density_profile(left, right, xs, x0, t, gam).mean(axis=-1)
