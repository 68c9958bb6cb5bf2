"""Exact solutions used to pin the oracle (test infrastructure only).

* ``advection``: u0(x - a t) on a periodic domain.
* ``burgers_characteristics``: before the first shock, u(x, t) = u0(xi) with
  xi + t u0(xi) = x, solved per point by safeguarded Newton iteration.
* ``riemann``: the exact Riemann solver for the Euler equations of a
  polytropic gas (the textbook construction of Toro, cited in Sec. 5.2 of the
  paper): the star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 with the
  shock (Rankine-Hugoniot) or rarefaction (isentropic) branch on each side,
  then the self-similar solution is sampled at x/t.
"""
from __future__ import annotations

import math

import numpy as np


def advection(u0, x, t, a=1.0, x_l=-1.0, x_r=1.0):
    L = x_r - x_l
    xs = np.mod(x - a * t - x_l, L) + x_l
    return u0(xs)


def burgers_characteristics(u0, du0, x, t, iters=60):
    """Solve xi + t u0(xi) = x for xi (valid while 1 + t u0'(xi) > 0)."""
    x = np.asarray(x, dtype=np.float64)
    xi = x - t * u0(x)
    for _ in range(iters):
        g = xi + t * u0(xi) - x
        dg = 1.0 + t * du0(xi)
        xi = xi - g / dg
    return u0(xi)


# ---------------------------------------------------------------- Riemann


def _side(p, rho, pk, ck, gamma):
    """Pressure function f_K and its derivative for one side."""
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    r = p / pk
    f = 2.0 * ck / (gamma - 1.0) * (r ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
    df = 1.0 / (rho * ck) * r ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def riemann_star(left, right, gamma=1.4, tol=1e-15):
    """Star-region pressure and velocity (p*, u*) of the Riemann problem."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    du = ur - ul
    if 2.0 * (cl + cr) / (gamma - 1.0) <= du:
        raise ValueError("vacuum is generated; not supported")
    # two-rarefaction estimate as the starting guess
    z = (gamma - 1.0) / (2.0 * gamma)
    p = ((cl + cr - 0.5 * (gamma - 1.0) * du) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(100):
        fl, dfl = _side(p, rl, pl, cl, gamma)
        fr, dfr = _side(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + du) / (dfl + dfr)
        if pn <= 0.0:
            pn = 0.5 * p
        change = abs(pn - p) / (0.5 * (pn + p))
        p = pn
        if change < tol:
            break
    fl, _ = _side(p, rl, pl, cl, gamma)
    fr, _ = _side(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(left, right, s, gamma=1.4):
    """Primitive state (rho, u, p) at similarity coordinate s = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = riemann_star(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for idx, si in np.ndenumerate(s):
        if si <= us:  # left of the contact
            c = math.sqrt(gamma * pl / rl)
            if ps > pl:  # left shock
                S = ul - c * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pl + (gamma - 1.0) / (2 * gamma))
                if si <= S:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                cs = c * (ps / pl) ** ((gamma - 1.0) / (2 * gamma))
                if si <= ul - c:
                    st = (rl, ul, pl)
                elif si >= us - cs:
                    st = (rl * (ps / pl) ** (1.0 / gamma), us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (c + 0.5 * (gamma - 1.0) * ul + si)
                    cc = 2.0 / (gamma + 1.0) * (c + 0.5 * (gamma - 1.0) * (ul - si))
                    rr_ = rl * (cc / c) ** (2.0 / (gamma - 1.0))
                    st = (rr_, uu, pl * (cc / c) ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            c = math.sqrt(gamma * pr / rr)
            if ps > pr:  # right shock
                S = ur + c * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pr + (gamma - 1.0) / (2 * gamma))
                if si >= S:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                cs = c * (ps / pr) ** ((gamma - 1.0) / (2 * gamma))
                if si >= ur + c:
                    st = (rr, ur, pr)
                elif si <= us + cs:
                    st = (rr * (ps / pr) ** (1.0 / gamma), us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (-c + 0.5 * (gamma - 1.0) * ur + si)
                    cc = 2.0 / (gamma + 1.0) * (c - 0.5 * (gamma - 1.0) * (ur - si))
                    rr_ = rr * (cc / c) ** (2.0 / (gamma - 1.0))
                    st = (rr_, uu, pr * (cc / c) ** (2.0 * gamma / (gamma - 1.0)))
        rho[idx], u[idx], p[idx] = st
    return rho, u, p
