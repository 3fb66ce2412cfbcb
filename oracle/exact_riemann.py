"""Exact Riemann solutions used to pin the oracle on the paper's shock tubes.

TEST INFRASTRUCTURE ONLY (part of the oracle).  The paper (Sec. 6.1.2, 6.1.3)
compares against exact solutions "computable from the initial data" without
printing a solver; these are written from the mathematics of the ideal-gas
Riemann problem.

Newtonian: the star-region pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0
with, for side K,
  shock (p > p_K):       f_K = (p - p_K) sqrt(A_K / (p + B_K)),
                         A_K = 2/((g+1) rho_K), B_K = (g-1)/(g+1) p_K;
  rarefaction (p <= p_K): f_K = 2 c_K/(g-1) [(p/p_K)^((g-1)/(2g)) - 1];
u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2; the self-similar profile then
follows from the Rankine-Hugoniot density ratio for shocks and from the
isentropic fan relations for rarefactions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fK(p, rho, pK, g):
    c = math.sqrt(g * pK / rho)
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        return (p - pK) * math.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def newtonian_star(rl, ul, pl, rr, ur, pr, g):
    """Star-region (p*, u*)."""
    f = lambda p: _fK(p, rl, pl, g) + _fK(p, rr, pr, g) + (ur - ul)
    hi = max(pl, pr)
    while f(hi) < 0.0:
        hi *= 2.0
    p = brentq(f, 1e-14 * min(pl, pr), hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    u = 0.5 * (ul + ur) + 0.5 * (_fK(p, rr, pr, g) - _fK(p, rl, pl, g))
    return p, u


def newtonian_sample(x, t, rl, ul, pl, rr, ur, pr, g, xd=0.0):
    """Primitive (rho, u, p) of the exact solution at positions x and time t > 0."""
    ps, us = newtonian_star(rl, ul, pl, rr, ur, pr, g)
    x = np.asarray(x, dtype=np.float64)
    rho = np.empty_like(x)
    u = np.empty_like(x)
    p = np.empty_like(x)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    for idx, xi in np.ndenumerate(x):
        s = (xi - xd) / t
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                SL = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s < SL:
                    r, v, q = rl, ul, pl
                else:
                    r, v, q = rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                head = ul - cl
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                tail = us - cs
                if s < head:
                    r, v, q = rl, ul, pl
                elif s > tail:
                    r, v, q = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    q = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                SR = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s > SR:
                    r, v, q = rr, ur, pr
                else:
                    r, v, q = rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
            else:  # right rarefaction
                head = ur + cr
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                tail = us + cs
                if s > head:
                    r, v, q = rr, ur, pr
                elif s < tail:
                    r, v, q = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    q = pr * (c / cr) ** (2.0 * g / (g - 1.0))
        rho[idx], u[idx], p[idx] = r, v, q
    return rho, u, p
