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


# ---------------------------------------------------------------------------
# Special-relativistic ideal gas, flow normal to the discontinuity (no tangential
# velocity), as in the shock tubes of tab:Riemann_Problems (Sec. 6.1.3).  Units
# with c = 1; h = 1 + g p / ((g - 1) rho), c_s^2 = g p / (rho h), W = 1/sqrt(1 - v^2).
#
# Rarefaction: the flow is isentropic (p = K rho^g) and, across a fan facing
# left (right), arctanh(v) + (-) (2/sqrt(g-1)) arctanh(c_s / sqrt(g-1)) is
# constant: with x = c_s / sqrt(g-1), p/rho is proportional to x^2/(1 - x^2) on
# the isentrope, so the integral of c_s d(rho)/rho is (2/sqrt(g-1)) arctanh(x).
# Inside the fan the characteristic speed (v -+ c_s)/(1 -+ v c_s) equals (x-x_d)/t.
#
# Shock: with [X] = X_b - X_a across the front (a ahead, b behind), the Taub
# adiabat [h^2] = [p](h_a/rho_a + h_b/rho_b) and the ideal-gas relation
# rho_b = g p_b / ((g-1)(h_b - 1)) give a quadratic for h_b,
#   (1 - q) h_b^2 + q h_b - h_a^2 - (p_b - p_a) h_a / rho_a = 0,
#   q = (g-1)(p_b - p_a)/(g p_b);
# the invariant mass flux is j^2 = -[p]/[h/rho]; for a front facing right,
#   V_s = (rho_a^2 W_a^2 v_a + j sqrt(j^2 + rho_a^2 W_a^2 (1 - v_a^2))) / (rho_a^2 W_a^2 + j^2),
#   v_b = (h_a W_a v_a + W_s [p]/j) / (h_a W_a + [p](W_s v_a / j + 1/(rho_a W_a))),
# with j > 0 and W_s = 1/sqrt(1 - V_s^2); a front facing left is its mirror image.
# The tests check these states against the Rankine-Hugoniot conditions and the
# whole solution against the integral conservation law.
# ---------------------------------------------------------------------------

def _sr_cs(rho, p, g):
    h = 1.0 + g * p / ((g - 1.0) * rho)
    return math.sqrt(g * p / (rho * h))


def _sr_rarefaction_left(rho_a, v_a, p_a, p_b, g):
    """State behind a left-facing fan from state a (on its left) down to p_b."""
    rho_b = rho_a * (p_b / p_a) ** (1.0 / g)
    s = math.sqrt(g - 1.0)
    ca, cb = _sr_cs(rho_a, p_a, g), _sr_cs(rho_b, p_b, g)
    y = math.atanh(v_a) + (2.0 / s) * (math.atanh(ca / s) - math.atanh(cb / s))
    return rho_b, math.tanh(y)


def _sr_shock_right(rho_a, v_a, p_a, p_b, g):
    """State behind a right-facing shock running into state a (on its right),
    and the shock speed."""
    h_a = 1.0 + g * p_a / ((g - 1.0) * rho_a)
    W_a = 1.0 / math.sqrt(1.0 - v_a * v_a)
    dp = p_b - p_a
    q = (g - 1.0) * dp / (g * p_b)
    A, B, C = 1.0 - q, q, -h_a * h_a - dp * h_a / rho_a
    h_b = (-B + math.sqrt(B * B - 4.0 * A * C)) / (2.0 * A)
    rho_b = g * p_b / ((g - 1.0) * (h_b - 1.0))
    j = math.sqrt(dp / (h_a / rho_a - h_b / rho_b))
    m2 = rho_a * rho_a * W_a * W_a
    V_s = (m2 * v_a + j * math.sqrt(j * j + m2 * (1.0 - v_a * v_a))) / (m2 + j * j)
    W_s = 1.0 / math.sqrt(1.0 - V_s * V_s)
    v_b = (h_a * W_a * v_a + W_s * dp / j) / (h_a * W_a + dp * (W_s * v_a / j + 1.0 / (rho_a * W_a)))
    return rho_b, v_b, V_s


def _sr_wave(side, rho_a, v_a, p_a, p, g):
    """(rho, v) behind the wave on `side` ('L' or 'R') that takes state a to
    pressure p, and the shock speed (None for a fan)."""
    if side == "R":
        if p > p_a:
            return _sr_shock_right(rho_a, v_a, p_a, p, g)
        rho_b, v_b = _sr_rarefaction_left(rho_a, -v_a, p_a, p, g)
        return rho_b, -v_b, None
    if p > p_a:
        rho_b, v_b, V_s = _sr_shock_right(rho_a, -v_a, p_a, p, g)
        return rho_b, -v_b, -V_s
    rho_b, v_b = _sr_rarefaction_left(rho_a, v_a, p_a, p, g)
    return rho_b, v_b, None


def sr_star(rl, vl, pl, rr, vr, pr, g):
    """Star-region pressure and velocity: the velocity behind the left wave, a
    decreasing function of p, equals that behind the right wave, an increasing one."""
    f = lambda p: _sr_wave("L", rl, vl, pl, p, g)[1] - _sr_wave("R", rr, vr, pr, p, g)[1]
    lo = 1e-12 * min(pl, pr)
    hi = max(pl, pr)
    while f(hi) > 0.0:
        hi *= 2.0
    p = brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
    return p, _sr_wave("L", rl, vl, pl, p, g)[1]


def sr_sample(x, t, rl, vl, pl, rr, vr, pr, g, xd=0.0):
    """Primitive (rho, v, p) of the exact solution at positions x and time t > 0,
    and the wave data (p*, v*, rho*_L, rho*_R, left and right shock speeds or None)."""
    ps, vs = sr_star(rl, vl, pl, rr, vr, pr, g)
    rsl, _, VL = _sr_wave("L", rl, vl, pl, ps, g)
    rsr, _, VR = _sr_wave("R", rr, vr, pr, ps, g)
    x = np.asarray(x, dtype=np.float64)
    rho, v, p = np.empty_like(x), np.empty_like(x), np.empty_like(x)

    def fan(side, s):
        # state inside a fan: the characteristic speed at pressure q equals s
        ra, va, pa = (rl, vl, pl) if side == "L" else (rr, vr, pr)

        def lam(q):
            rq, vq, _ = _sr_wave(side, ra, va, pa, q, g)
            c = _sr_cs(rq, q, g)
            return (vq - c) / (1.0 - vq * c) if side == "L" else (vq + c) / (1.0 + vq * c)

        q = brentq(lambda q: lam(q) - s, ps, pa, xtol=1e-300, rtol=1e-15, maxiter=500)
        rq, vq, _ = _sr_wave(side, ra, va, pa, q, g)
        return rq, vq, q

    for idx, xi in np.ndenumerate(x):
        s = (xi - xd) / t
        if s <= vs:
            if VL is not None:
                st = (rl, vl, pl) if s < VL else (rsl, vs, ps)
            else:
                cl, csl = _sr_cs(rl, pl, g), _sr_cs(rsl, ps, g)
                head, tail = (vl - cl) / (1.0 - vl * cl), (vs - csl) / (1.0 - vs * csl)
                st = (rl, vl, pl) if s < head else ((rsl, vs, ps) if s > tail else fan("L", s))
        else:
            if VR is not None:
                st = (rr, vr, pr) if s > VR else (rsr, vs, ps)
            else:
                cr, csr = _sr_cs(rr, pr, g), _sr_cs(rsr, ps, g)
                head, tail = (vr + cr) / (1.0 + vr * cr), (vs + csr) / (1.0 + vs * csr)
                st = (rr, vr, pr) if s > head else ((rsr, vs, ps) if s < tail else fan("R", s))
        rho[idx], v[idx], p[idx] = st
    return (rho, v, p), (ps, vs, rsl, rsr, VL, VR)
