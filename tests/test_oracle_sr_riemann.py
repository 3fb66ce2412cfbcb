"""Pins of the special-relativistic exact Riemann solver (oracle/exact_riemann.py)
and, through it, of the oracle's SR shock path on the paper's shock tubes
(tab:Riemann_Problems, Sec. 6.1.3, tab:RE_sod).

The solver is checked against the physics, not against itself: the shock states
satisfy the relativistic Rankine-Hugoniot conditions, the whole solution (fans
included) satisfies the integral conservation law, the Newtonian limit agrees
with the Newtonian exact solver, and the wave data match what Sec. 6.1.3 states
about the two shock tubes."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import dg_inputs as di
import oracle
from oracle import exact_riemann as ex
from tests.conftest import read_golden


def _cons_flux(rho, v, p, g):
    """SR conserved variables (D, S, tau) and their x fluxes for flow along x."""
    W = 1.0 / math.sqrt(1.0 - v * v)
    h = 1.0 + g * p / ((g - 1.0) * rho)
    D, S = rho * W, rho * h * W * W * v
    tau = rho * h * W * W - p - D
    return np.array([D, S, tau]), np.array([D * v, S * v + p, S - D * v])


def _cs(rho, p, g):
    h = 1.0 + g * p / ((g - 1.0) * rho)
    return math.sqrt(g * p / (rho * h))


CASES = {"st1": di.RIEMANN["st1"], "st2": di.RIEMANN["st2"],
         # mirror image of shock tube 1: a left-facing shock and a right-facing fan
         "st1_mirror": (1.0, 0.0, 1e-8, 10.0, 0.0, 13.33, 5.0 / 3.0, 0.5),
         # both waves shocks: two streams colliding
         "collision": (1.0, 0.6, 1.0, 1.0, -0.6, 1.0, 5.0 / 3.0, 0.5)}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sr_shocks_satisfy_rankine_hugoniot(name):
    """[F] = V_s [U] across every shock of the solution, for D, S and tau."""
    rl, vl, pl, rr, vr, pr, g, xd = CASES[name]
    _, (ps, vs, rsl, rsr, VL, VR) = ex.sr_sample([xd], 1.0, rl, vl, pl, rr, vr, pr, g, xd)
    shocks = [(VL, (rl, vl, pl), (rsl, vs, ps)), (VR, (rsr, vs, ps), (rr, vr, pr))]
    checked = 0
    for V, a, b in shocks:
        if V is None:
            continue
        Ua, Fa = _cons_flux(*a, g)
        Ub, Fb = _cons_flux(*b, g)
        scale = np.abs(Ua).max() + np.abs(Ub).max() + np.abs(Fa).max() + np.abs(Fb).max()
        assert np.all(np.abs((Fb - Fa) - V * (Ub - Ua)) <= 1e-11 * scale), (name, V)
        checked += 1
    assert checked == {"st1": 1, "st2": 1, "st1_mirror": 1, "collision": 2}[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_sr_exact_solution_conserves(name):
    """The integral of (D, S, tau) over [x_d - 1, x_d + 1] grows by T (F_L - F_R)
    between t = 0 and t = T: the constant pieces integrate exactly and each fan
    by adaptive quadrature, so every wave speed, star state and fan profile
    enters."""
    rl, vl, pl, rr, vr, pr, g, xd = CASES[name]
    T = 0.4
    _, (ps, vs, rsl, rsr, VL, VR) = ex.sr_sample([xd], T, rl, vl, pl, rr, vr, pr, g, xd)
    UL, FL = _cons_flux(rl, vl, pl, g)
    UR, FR = _cons_flux(rr, vr, pr, g)
    Usl, _ = _cons_flux(rsl, vs, ps, g)
    Usr, _ = _cons_flux(rsr, vs, ps, g)
    a, b = xd - 1.0, xd + 1.0

    def U_at(x):
        (r, v, p), _ = ex.sr_sample([x], T, rl, vl, pl, rr, vr, pr, g, xd)
        return _cons_flux(r[0], v[0], p[0], g)[0]

    def fan_integral(x0, x1):
        return np.array([quad(lambda x: U_at(x)[k], x0, x1, epsabs=0, epsrel=1e-12, limit=200)[0]
                         for k in range(3)])

    total = np.zeros(3)
    # left wave
    if VL is not None:
        xl = xd + VL * T
        total += UL * (xl - a)
        xs = xl
    else:
        cl, csl = _cs(rl, pl, g), _cs(rsl, ps, g)
        xh, xt = xd + T * (vl - cl) / (1 - vl * cl), xd + T * (vs - csl) / (1 - vs * csl)
        total += UL * (xh - a) + fan_integral(xh, xt)
        xs = xt
    xc = xd + vs * T
    total += Usl * (xc - xs)
    # right wave
    if VR is not None:
        xr = xd + VR * T
        total += Usr * (xr - xc) + UR * (b - xr)
    else:
        cr, csr = _cs(rr, pr, g), _cs(rsr, ps, g)
        xt, xh = xd + T * (vs + csr) / (1 + vs * csr), xd + T * (vr + cr) / (1 + vr * cr)
        total += Usr * (xt - xc) + fan_integral(xt, xh) + UR * (b - xh)
    expected = UL * (xd - a) + UR * (b - xd) + T * (FL - FR)
    assert np.all(np.abs(total - expected) <= 1e-9 * np.abs(expected).max()), (name, total, expected)


def test_sr_newtonian_limit():
    """Shock tube 1 with its pressures scaled by 1e-8: the SR star state tends to
    the Newtonian one (relative differences of the order of p/rho)."""
    rl, vl, pl, rr, vr, pr, g, xd = di.RIEMANN["st1"]
    eps = 1e-8
    ps, vs = ex.sr_star(rl, vl, pl * eps, rr, vr, pr * eps, g)
    pn, un = ex.newtonian_star(rl, vl, pl * eps, rr, vr, pr * eps, g)
    assert abs(ps / pn - 1.0) < 1e-6 and abs(vs / un - 1.0) < 1e-6, (ps, pn, vs, un)


def test_sr_shock_tubes_match_the_papers_description():
    """Sec. 6.1.3: in shock tube 1 the flow reaches a mildly relativistic speed of
    about 0.7; in shock tube 2 the shock moves at about 0.986 (a Lorentz factor of
    about 6) and the dense shell between contact and shock is about 0.01 wide at
    t = 0.4."""
    _, (ps, vs, *_rest) = ex.sr_sample([0.5], 0.4, *di.RIEMANN["st1"])
    assert 0.69 < vs < 0.74, vs
    _, (ps2, vs2, rsl2, rsr2, VL2, VR2) = ex.sr_sample([0.5], 0.4, *di.RIEMANN["st2"])
    assert VL2 is None and abs(VR2 - 0.986) < 0.002, VR2
    assert 5.5 < 1.0 / math.sqrt(1.0 - VR2 ** 2) < 6.5
    assert 0.009 < (VR2 - vs2) * 0.4 < 0.012


def _st_relative_error(name, nx, n=2, flux=1, limiter=2, cfl=0.2, T=0.4):
    # x in [0, 1] (x_d = 0.5) is embedded in a periodic [0, 2] holding the mirror
    # image about x = 1; no wave from the mirror problem or the wrap enters [0, 1]
    # before T = 0.4 (fastest speeds: shock tube 1, 0.83 to the right and 0.72 to
    # the left; shock tube 2, 0.987 and 0.82).
    spec = oracle.MeshSpec(system=1, dim=1, K=(2 * nx, 1, 1), n=n, flux=flux, limiter=limiter, gamma=5.0 / 3.0,
                           lo=(0, 0, 0), hi=(2, 1, 1))
    m = oracle.Mesh(spec)
    x = m.coords()[0]
    rl, vl, pl, rr, vr, pr, g, xd = di.RIEMANN[name]
    left = (x <= xd) | (x > 2.0 - xd)
    z = np.zeros_like(x)
    U = m.from_prim(np.stack([np.where(left, rl, rr), z, z, z, np.where(left, pl, pr)]))
    t = 0.0
    while t < T - 1e-15:
        h = min(m.cfl_dt(U, cfl), T - t)
        U = m.rk3_step(U, h)
        t += h
    (rho, v, p), _ = ex.sr_sample(x, T, rl, vl, pl, rr, vr, pr, g, xd)
    Uex = m.from_prim(np.stack([rho, v, z, z, p]))
    _, w = oracle.lgl(n)
    inside = x.reshape(m.E, m.nn).mean(axis=1) < 1.0
    err = (np.abs(U - Uex)[inside] * w[None, None, :]).sum() / (2 * nx)
    norm = (np.abs(Uex)[inside] * w[None, None, :]).sum() / (2 * nx)
    return err / norm, norm


def test_re_sod_st1_table_loose():
    """tab:RE_sod, shock tube 1, HLL-MinMod-2: the relative L1 errors within the
    band the unstated time step and exterior states allow (0.6-1.2x the printed
    values), local orders near 1, and the normalisation near the caption's 21."""
    rows = read_golden("re_sod_st1_hll_minmod2.txt")
    res = [_st_relative_error("st1", int(nx)) for nx, _ in rows]
    for (nx, ref), (e, norm) in zip(rows, res):
        assert 0.6 * ref < e < 1.2 * ref, (nx, e, ref)
        assert abs(norm - 21.0) < 0.5, norm
    for i in range(len(res) - 1):
        o = math.log2(res[i][0] / res[i + 1][0])
        assert 0.5 < o < 1.25, (res, o)


def test_planted_errors_in_the_exact_solver_are_caught(monkeypatch):
    """The solver pins reject a fan invariant with the wrong factor (1 for
    2/sqrt(g-1)) and a shock speed off by 1 %: planted in the solver on the CPU."""
    good_fan, good_shock = ex._sr_rarefaction_left, ex._sr_shock_right

    def bad_fan(rho_a, v_a, p_a, p_b, g):
        rho_b = rho_a * (p_b / p_a) ** (1.0 / g)
        s = math.sqrt(g - 1.0)
        ca, cb = _cs(rho_a, p_a, g), _cs(rho_b, p_b, g)
        return rho_b, math.tanh(math.atanh(v_a) + (1.0 / s) * (math.atanh(ca / s) - math.atanh(cb / s)))

    def bad_shock(rho_a, v_a, p_a, p_b, g):
        rho_b, v_b, V_s = good_shock(rho_a, v_a, p_a, p_b, g)
        return rho_b, v_b, 1.01 * V_s

    for name in ("st1", "st1_mirror", "st2"):
        monkeypatch.setattr(ex, "_sr_rarefaction_left", bad_fan)
        with pytest.raises(AssertionError):
            test_sr_exact_solution_conserves(name)
        monkeypatch.setattr(ex, "_sr_rarefaction_left", good_fan)
    monkeypatch.setattr(ex, "_sr_shock_right", bad_shock)
    for name in sorted(CASES):
        with pytest.raises(AssertionError):
            test_sr_shocks_satisfy_rankine_hugoniot(name)
        with pytest.raises(AssertionError):
            test_sr_exact_solution_conserves(name)


def test_re_sod_st2_table_loose():
    """tab:RE_sod, shock tube 2, LLF-MinMod-2: the printed order (about 0.7, "a bit
    lower than first order") and the caption's normalisation (about 1,151); the
    errors come out 1.4-1.5x the printed ones at C = 0.2 and move with the time
    step (2.2x at C = 0.1), which the paper does not give, so the band is wide."""
    rows = read_golden("re_sod_st2_llf_minmod2.txt")
    res = [_st_relative_error("st2", int(nx), flux=0) for nx, _ in rows]
    for (nx, ref), (e, norm) in zip(rows, res):
        assert 0.6 * ref < e < 1.7 * ref, (nx, e, ref)
        assert abs(norm - 1151.0) < 5.0, norm
    for i in range(len(res) - 1):
        o = math.log2(res[i][0] / res[i + 1][0])
        assert 0.5 < o < 0.9, (res, o)
