"""Pins of the oracle's point-wise physics: primitive recovery (Sec. 2.1.1,
2.1.2), characteristic speeds (eq:CharDecomp) and the numerical fluxes
(eq:LLF, eq:HLL)."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import dg_inputs as di
import oracle


def test_c2p_static_closed_form():
    # v = 0: W = 1, rho = D and p = (gamma - 1) tau exactly
    g = 4.0 / 3.0
    cons = np.array([[2.0, 0.1], [0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [3.0, 1e-7]])
    prim, it, st = oracle.con2prim(g, cons)
    assert np.all(st == 0)
    assert np.array_equal(prim[0], cons[0])
    assert np.array_equal(prim[4], (g - 1.0) * cons[4])
    assert np.all(it == 1)


def test_c2p_round_trip_conditioned():
    g = 4.0 / 3.0
    prim = di.c2p_samples(11, 50000, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    out, it, st = oracle.con2prim(g, cons)
    assert np.all(st == 0)
    kappa = cons[4] / (prim[4] / (g - 1.0))  # tau / (rho eps): amplification of input rounding
    for v in (0, 1, 2, 3, 4):
        scale = np.maximum(np.abs(prim[v]), 1e-300) if v in (0, 4) else np.sqrt(
            prim[1] ** 2 + prim[2] ** 2 + prim[3] ** 2) + 1e-300
        rel = np.abs(out[v] - prim[v]) / scale
        assert np.all(rel <= 1e-14 * (1.0 + kappa)), (v, (rel / (1 + kappa)).max())
    well = kappa < 1e2
    assert np.all(np.abs(out[4] - prim[4])[well] / prim[4][well] <= 1e-12)


def test_c2p_newton_converges_quadratically():
    """Sec. 2.1.2 con2prim: Newton on f(p) with the exact f'(p).  From a guess 0.1 % off the
    root, well-conditioned states (tau/(rho eps) < 10) stop within five
    iterations (the error squares each step; the stopping rule adds one step);
    a wrong derivative would converge only linearly."""
    g = 4.0 / 3.0
    prim = di.c2p_samples(12, 20000, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    kappa = cons[4] / (prim[4] / (g - 1.0))
    _, it, st = oracle.con2prim(g, cons, guess=prim[4] * (1.0 + 1e-3))
    well = kappa < 10
    assert np.all(st == 0) and well.sum() > 1000
    assert it[well].max() <= 5 and np.median(it[well]) <= 4, np.bincount(it[well])


def _c2p_zroot(g, D, S, tau):
    """Independent reference: 1D root in z = W v (Galeazzi-type formulation),
    with q = tau/D, r = |S|/D, eps(z) = W q - z r + z^2/(1+W), h = 1 + g eps."""
    q, r = tau / D, S / D

    def eps(z):
        W = math.sqrt(1.0 + z * z)
        return W * q - z * r + z * z / (1.0 + W)

    def f(z):
        return z - r / (1.0 + g * max(eps(z), 0.0))

    if r == 0.0:
        z = 0.0
    else:
        z = brentq(f, 0.0, r, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=400)
    W = math.sqrt(1.0 + z * z)
    rho = D / W
    return rho, (g - 1.0) * rho * eps(z)


def test_c2p_matches_independent_z_root():
    g = 4.0 / 3.0
    prim = di.c2p_samples(5, 3000, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    out, _, st = oracle.con2prim(g, cons)
    assert np.all(st == 0)
    kappa = cons[4] / (prim[4] / (g - 1.0))
    sel = np.nonzero(kappa < 1e2)[0][:600]
    assert sel.size > 100
    for q in sel:
        S = math.sqrt(cons[1, q] ** 2 + cons[2, q] ** 2 + cons[3, q] ** 2)
        rho, p = _c2p_zroot(g, cons[0, q], S, cons[4, q])
        assert abs(out[0, q] - rho) <= 1e-13 * rho
        assert abs(out[4, q] - p) <= 1e-13 * p


def test_c2p_rejects_unphysical():
    g = 4.0 / 3.0
    cons = np.array([[-1.0, 1.0, 1.0], [0.0, 0.0, 5.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0],
                     [1.0, -1.0, 1.0]])
    _, _, st = oracle.con2prim(g, cons)
    assert list(st) == [1, 1, 1]  # D <= 0; tau <= 0; S^2 >= tau (tau + 2 D)


@pytest.mark.parametrize("system,gamma,flux", [(0, 1.4, 0), (0, 1.4, 1), (0, 1.4, 2), (1, 4.0 / 3.0, 0),
                                               (1, 4.0 / 3.0, 1)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flux_consistency(system, gamma, flux, axis):
    # F*(U, U) = F(U) (Sec. 3.2)
    prim = np.array([[1.3], [0.2], [-0.4], [0.1], [0.7]])
    u = oracle.prim2con(system, gamma, prim)[:, 0]
    Fs, FL, FR, _ = oracle.num_flux(system, gamma, flux, axis, u, u)
    assert np.allclose(Fs, FL, rtol=1e-15, atol=1e-15)
    # and the physical flux is the textbook one
    rho, v, p = prim[0, 0], prim[1:4, 0], prim[4, 0]
    if system == 0:
        E = p / (gamma - 1) + 0.5 * rho * v @ v
        ref = [rho * v[axis]] + [rho * v[i] * v[axis] + p * (i == axis) for i in range(3)] + [(E + p) * v[axis]]
    else:
        W = 1 / math.sqrt(1 - v @ v)
        h = 1 + gamma / (gamma - 1) * p / rho
        D, S, tau = rho * W, rho * h * W * W * v, rho * h * W * W - p - rho * W
        ref = [D * v[axis]] + [S[i] * v[axis] + p * (i == axis) for i in range(3)] + [(tau + p) * v[axis]]
    assert np.allclose(FL, ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("system,gamma,vx", [(0, 1.4, 3.0), (1, 4.0 / 3.0, 0.95)])
def test_hll_reduces_to_upwind(system, gamma, vx):
    # supersonic flow along +x: c_min = 0, so HLL = F(U_L) (Sec. 3.2.2)
    pl = np.array([[1.0], [vx], [0.0], [0.0], [0.1]])
    pr = np.array([[0.5], [vx * 0.9], [0.0], [0.0], [0.05]])
    uL = oracle.prim2con(system, gamma, pl)[:, 0]
    uR = oracle.prim2con(system, gamma, pr)[:, 0]
    Fs, FL, FR, sp = oracle.num_flux(system, gamma, 1, 0, uL, uR)
    assert sp[0] > 0 and sp[2] > 0
    assert np.allclose(Fs, FL, rtol=1e-14, atol=1e-15)
    # and upwinding from the right when everything moves left
    Fs2, FL2, FR2, sp2 = oracle.num_flux(system, gamma, 1, 0, uR * np.array([1, -1, 1, 1, 1]),
                                         uL * np.array([1, -1, 1, 1, 1]))
    assert np.allclose(Fs2, FR2, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("system,gamma", [(0, 1.4), (1, 4.0 / 3.0)])
def test_llf_equals_hll_for_symmetric_speeds(system, gamma):
    # static states with equal sound speed but different density and pressure
    # (p / rho fixed, so c^2 = g p / rho, and in SR h and c_s, agree): c_max =
    # -c_min = alpha, and then the HLL formula is algebraically the LLF one,
    # dissipation term included (the jump U_R - U_L is not zero)
    pl = np.array([[1.0], [0.0], [0.0], [0.0], [1.0]])
    pr = np.array([[2.0], [0.0], [0.0], [0.0], [2.0]])
    uL = oracle.prim2con(system, gamma, pl)[:, 0]
    uR = oracle.prim2con(system, gamma, pr)[:, 0]
    F0, FL, FR, sp = oracle.num_flux(system, gamma, 0, 1, uL, uR)
    F1, *_ = oracle.num_flux(system, gamma, 1, 1, uL, uR)
    assert sp[0] == -sp[1] and abs(sp[1] - sp[3]) <= 1e-15 * sp[1]
    assert np.abs(F0 - 0.5 * (FL + FR)).max() > 0.1  # the dissipation term is in play
    assert np.allclose(F0, F1, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("system,gamma,flux", [(0, 1.4, 0), (0, 1.4, 1), (0, 1.4, 2), (1, 4.0 / 3.0, 0),
                                               (1, 4.0 / 3.0, 1)])
def test_numerical_flux_mirror_symmetry(system, gamma, flux):
    """The numerical fluxes of Sec. 3.2 treat both sides alike: mirroring x -> -x
    (swap the states, flip their x momenta) flips the flux, F*(R u_R, R u_L) =
    -R F*(u_L, u_R) with R = diag(1, -1, 1, 1, 1).  The states differ in density,
    pressure and velocity, so each side has its own speeds."""
    pl = np.array([[1.0], [0.3], [0.1], [0.0], [1.0]])
    pr = np.array([[0.4], [-0.5], [0.2], [0.1], [0.3]]) if system == 0 else \
        np.array([[0.4], [-0.6], [0.2], [0.1], [0.3]])
    uL = oracle.prim2con(system, gamma, pl)[:, 0]
    uR = oracle.prim2con(system, gamma, pr)[:, 0]
    R = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    Fs, _, _, sp = oracle.num_flux(system, gamma, flux, 0, uL, uR)
    Fm, _, _, _ = oracle.num_flux(system, gamma, flux, 0, R * uR, R * uL)
    assert max(abs(sp[0]), abs(sp[1])) != max(abs(sp[2]), abs(sp[3]))
    assert np.allclose(Fm, -R * Fs, rtol=1e-13, atol=1e-14), (Fm, -R * Fs)


def test_sr_speeds_limits():
    # at v = 0 the SR speeds are -+cs with cs^2 = g p / (rho h)
    g = 4.0 / 3.0
    rho, p = 2.0, 0.5
    u = oracle.prim2con(1, g, np.array([[rho], [0.0], [0.0], [0.0], [p]]))[:, 0]
    _, _, _, sp = oracle.num_flux(1, g, 1, 0, u, u)
    h = 1 + g / (g - 1) * p / rho
    cs = math.sqrt(g * p / (rho * h))
    assert np.allclose(sp[:2], [-cs, cs], rtol=1e-14)
    # relativistic velocity addition along the flow direction
    v = 0.6
    u = oracle.prim2con(1, g, np.array([[rho], [v], [0.0], [0.0], [p]]))[:, 0]
    _, _, _, sp = oracle.num_flux(1, g, 1, 0, u, u)
    assert np.allclose(sp[:2], [(v - cs) / (1 - v * cs), (v + cs) / (1 + v * cs)], rtol=1e-13)


def _euler_jacobian(g, vel, H, axis):
    """Analytic flux Jacobian dF^axis/dU of the 3D Euler equations (ideal gas) at
    velocity vel and specific enthalpy H (textbook form, written out here)."""
    q2 = vel @ vel
    un = vel[axis]
    A = np.zeros((5, 5))
    A[0, 1 + axis] = 1.0
    for i in range(3):
        A[1 + i, 0] = -vel[i] * un
        A[1 + i, 1 + i] += un
        A[1 + i, 1 + axis] += vel[i]
    A[1 + axis, 0] += 0.5 * (g - 1.0) * q2
    for j in range(3):
        A[1 + axis, 1 + j] -= (g - 1.0) * vel[j]
    A[1 + axis, 4] = g - 1.0
    A[4, 0] = un * (0.5 * (g - 1.0) * q2 - H)
    for j in range(3):
        A[4, 1 + j] = -(g - 1.0) * un * vel[j]
    A[4, 1 + axis] += H
    A[4, 4] = g * un
    return A


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_roe_flux_matches_eigendecomposition(axis):
    """eq:Roe for the ideal gas equals 1/2 (F_L + F_R) - 1/2 |A| (U_R - U_L) with A
    the analytic Jacobian at the Roe averages (eq:RoeAverages) and |A| formed
    from a numerical eigendecomposition; and A (U_R - U_L) = F_R - F_L (Roe's
    conservation condition)."""
    g = 1.4
    pl = np.array([[1.0], [0.75], [0.1], [-0.2], [1.0]])
    pr = np.array([[0.125], [0.05], [0.3], [0.05], [0.1]])
    uL = oracle.prim2con(0, g, pl)[:, 0]
    uR = oracle.prim2con(0, g, pr)[:, 0]
    Fs, FL, FR, _ = oracle.num_flux(0, g, 2, axis, uL, uR)
    sl, sr = math.sqrt(pl[0, 0]), math.sqrt(pr[0, 0])
    vel = (sl * pl[1:4, 0] + sr * pr[1:4, 0]) / (sl + sr)
    hL = (uL[4] + pl[4, 0]) / pl[0, 0]
    hR = (uR[4] + pr[4, 0]) / pr[0, 0]
    H = (sl * hL + sr * hR) / (sl + sr)
    A = _euler_jacobian(g, vel, H, axis)
    assert np.allclose(A @ (uR - uL), FR - FL, rtol=1e-13, atol=1e-13)
    lam, R = np.linalg.eig(A)
    absA = (R * np.abs(lam.real)) @ np.linalg.inv(R)
    ref = 0.5 * (FL + FR) - 0.5 * absA.real @ (uR - uL)
    assert np.allclose(Fs, ref, rtol=1e-12, atol=1e-13), (Fs, ref)


def test_roe_upwinds_supersonic_flow():
    """All Roe eigenvalues of one sign: eq:Roe is the upwind flux."""
    g = 1.4
    pl = np.array([[1.0], [3.0], [0.2], [0.0], [0.1]])
    pr = np.array([[0.5], [2.8], [-0.1], [0.1], [0.05]])
    uL = oracle.prim2con(0, g, pl)[:, 0]
    uR = oracle.prim2con(0, g, pr)[:, 0]
    Fs, FL, FR, _ = oracle.num_flux(0, g, 2, 0, uL, uR)
    assert np.allclose(Fs, FL, rtol=1e-13, atol=1e-14)
    flip = np.array([1, -1, 1, 1, 1])
    Fs2, FL2, FR2, _ = oracle.num_flux(0, g, 2, 0, uR * flip, uL * flip)
    assert np.allclose(Fs2, FR2, rtol=1e-13, atol=1e-14)


def test_roe_is_newtonian_only():
    with pytest.raises(Exception):
        oracle.Mesh(oracle.MeshSpec(system=1, K=(2, 2, 2), n=3, flux=2, gamma=4.0 / 3.0))
