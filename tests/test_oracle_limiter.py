"""Pins of the oracle's limiters (Sec. 3.3.1 minmod / minmodB, Sec. 3.3.2 the
generalized high-order detector)."""
import numpy as np
import pytest

import dg_inputs as di
import oracle


def _linear_state(m, coefs):
    x, y, z = m.coords()
    U = np.empty((m.E, 5, m.nn))
    for v in range(5):
        a, b, c, d = coefs[v]
        U[:, v, :] = (a + b * x + c * y + d * z).reshape(m.E, m.nn)
    return U


@pytest.mark.parametrize("n", [2, 3, 5])
def test_linear_data_not_limited(n):
    """A linear solution is never modified (the detector passes it; Sec. 3.3.2).
    Elements next to the periodic wrap see a jump and are excluded."""
    K = 5
    m = oracle.Mesh(oracle.MeshSpec(system=0, K=(K, K, K), n=n, limiter=1))
    coefs = [(3.0, 0.5, -0.2, 0.1), (0.1, 1.0, 0.0, 0.0), (0.0, 0.0, 2.0, 0.0), (0.2, 0.0, 0.0, -1.0),
             (5.0, 0.3, 0.3, 0.3)]
    U = _linear_state(m, coefs)
    L, t = m.limit(U)
    e = np.arange(m.E)
    ex, ey, ez = e % K, (e // K) % K, e // (K * K)
    interior = (ex > 0) & (ex < K - 1) & (ey > 0) & (ey < K - 1) & (ez > 0) & (ez < K - 1)
    assert np.all(t[interior] == 0)
    assert np.array_equal(L[interior], U[interior])


@pytest.mark.parametrize("limiter", [1, 2])
def test_limiter_keeps_cell_means(limiter):
    m = oracle.Mesh(oracle.MeshSpec(system=1, K=(4, 4, 4), n=4, limiter=limiter, gamma=4 / 3))
    U = m.from_prim(di.blast_sr(m.coords(), seed=3))
    S0 = m.summaries(U)[:, :, 0]
    L, t = m.limit(U)
    assert t.any()
    S1 = m.summaries(L)[:, :, 0]
    assert np.allclose(S1, S0, rtol=1e-14, atol=1e-15)


def test_minmod_hand_case():
    """1D, N = 1, three elements with means (0, 1, 3) and a steep middle slope:
    plain minmod (beta = 2) limits the middle slope to
    m(U_x, (3-1)/(dx/2), (1-0)/(dx/2)) = 2/dx."""
    dx = 1.0 / 3.0
    m = oracle.Mesh(oracle.MeshSpec(system=0, dim=1, K=(3, 1, 1), n=2, limiter=2))
    U = np.zeros((3, 5, 2))
    means = [1.0, 1.0 + 1.0, 1.0 + 3.0]  # positive density; offsets 0, 1, 3
    slope_mid = 50.0
    for e in range(3):
        s = slope_mid if e == 1 else 0.0
        U[e, :, 0] = means[e] - 0.5 * dx * s
        U[e, :, 1] = means[e] + 0.5 * dx * s
    L, t = m.limit(U)
    a = 2.0 / dx
    assert np.allclose(L[1, 0], [means[1] - 0.5 * dx * a, means[1] + 0.5 * dx * a], rtol=1e-14)
    # first element: its own slope is 0 -> minmod = 0 (sign(0) = 0)
    assert np.allclose(L[0, 0], [means[0], means[0]], rtol=1e-15)
    # opposite signs of the three estimates give zero slope
    U2 = U.copy()
    U2[1, :, 0], U2[1, :, 1] = means[1] + 0.5 * dx * slope_mid, means[1] - 0.5 * dx * slope_mid
    L2, _ = m.limit(U2)
    assert np.allclose(L2[1, 0], [means[1], means[1]], rtol=1e-15)


def test_minmodB_M_keeps_small_slopes():
    """m_B returns a1 when |a1| <= M dx^2 (eq:MinModB)."""
    dx = 1.0 / 3.0
    m = oracle.Mesh(oracle.MeshSpec(system=0, dim=1, K=(3, 1, 1), n=2, limiter=2, tvb_M=1e4))
    U = np.zeros((3, 5, 2))
    for e in range(3):
        s = 5.0 if e == 1 else 0.0
        U[e, :, 0] = 1.0 - 0.5 * dx * s
        U[e, :, 1] = 1.0 + 0.5 * dx * s
    L, _ = m.limit(U)
    assert np.allclose(L, U, rtol=1e-14)


@pytest.mark.parametrize("n,limiter", [(2, 2), (3, 1), (4, 1)])
def test_tvd_in_the_means(n, limiter):
    """M = 0: no new extrema in the cell means (Sec. 3.3.1).  A density pulse in
    uniform velocity and pressure is a passive scalar, for which the property holds."""
    K = 24
    m = oracle.Mesh(oracle.MeshSpec(system=0, dim=1, K=(K, 1, 1), n=n, flux=1, limiter=limiter))
    x = m.coords()
    rho = np.where(np.abs(x[0] - 0.5) < 0.2, 2.0, 1.0)
    prim = np.stack([rho, np.full_like(rho, 1.0), 0 * rho, 0 * rho, np.full_like(rho, 1.0)])
    U = m.from_prim(prim)
    U, _ = m.limit(U)
    means = m.summaries(U)[:, 0, 0]
    hi, lo = means.max(), means.min()
    # the high-order detector leaves deviations below its 1e-8 tolerance alone
    slack = 1e-12 if limiter == 2 else 1e-8
    for _ in range(30):
        U = m.rk3_step(U, 0.5 * m.cfl_dt(U, 0.2))
        means = m.summaries(U)[:, 0, 0]
        assert means.max() <= hi + slack and means.min() >= lo - slack
        hi, lo = means.max(), means.min()


def test_unphysical_cells_always_limited():
    """SR: an element holding an unphysical node is limited in every variable (Sec. 3.3)."""
    m = oracle.Mesh(oracle.MeshSpec(system=1, K=(3, 3, 3), n=3, limiter=1, gamma=4 / 3))
    prim = np.stack([np.ones(m.E * m.nn), np.zeros(m.E * m.nn), np.zeros(m.E * m.nn),
                     np.zeros(m.E * m.nn), np.ones(m.E * m.nn)])
    U = m.from_prim(prim)
    U[13, 4, 5] = -1.0  # tau < 0 at one node of the centre element
    _, t = m.limit(U)
    assert t[13] == 0b11111
    assert np.count_nonzero(t) >= 1


def test_fix_bounds():
    """Sec. 2.1.4 reading: D >= D_atm, tau >= tau_atm D, S^2 <= (1 - 1e-12) tau (tau + 2 D)."""
    m = oracle.Mesh(oracle.MeshSpec(system=1, K=(1, 1, 1), n=2, gamma=4 / 3))
    U = np.zeros((1, 5, 8))
    U[0, 0] = [1.0, -1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    U[0, 4] = [1.0, 1.0, -5.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    U[0, 1] = [0.0, 0.0, 0.0, 10.0, 0.0, 0.0, 0.0, 0.0]
    F, nchg = m.fix(U)
    assert nchg == 3
    D, tau = F[0, 0], F[0, 4]
    s2 = F[0, 1] ** 2 + F[0, 2] ** 2 + F[0, 3] ** 2
    assert np.all(D >= 1e-12) and np.all(tau >= 1e-14 * D)
    bound = (1 - 1e-12) * tau * (tau + 2 * D)
    assert np.all(s2 <= bound * (1 + 1e-15))
    # the rescaled momentum sits on the bound (the fix takes no more than it must)
    assert abs(s2[3] / bound[3] - 1) < 2e-15 and np.array_equal(F[0, 1:4, :3], U[0, 1:4, :3])
    _, _, st = oracle.con2prim(4 / 3, F[0])
    assert np.all(st == 0)


def _mrs_mesh(K, n, alpha, dim=1):
    Ks = (K, 1, 1) if dim == 1 else (K, K, K)
    return oracle.Mesh(oracle.MeshSpec(system=0, dim=dim, K=Ks, n=n, flux=2, limiter=3, gamma=1.4,
                                       mrs_alpha=alpha))


def test_mrs_rescales_with_one_theta_and_keeps_means():
    """eq:MRSSol: every element becomes U0 + Theta (U - U0) with a single Theta in
    [0, 1] for all conserved variables and nodes; the cell means are kept."""
    m = _mrs_mesh(3, 4, 0.5, dim=3)
    U = m.from_prim(di.kh_ne(m.coords(), seed=4, amp=0.3))
    V, t = m.limit(U)
    S0 = m.summaries(U)[:, :, 0]
    S1 = m.summaries(V)[:, :, 0]
    assert np.allclose(S0, S1, rtol=0, atol=1e-14 * np.abs(S0).max())
    assert (t != 0).any()
    for e in range(m.E):
        d0 = U[e] - S0[e][:, None]
        d1 = V[e] - S0[e][:, None]
        big = np.abs(d0) > 1e-12 * np.abs(U[e]).max()
        th = d1[big] / d0[big]
        assert np.all((th >= -1e-12) & (th <= 1 + 1e-12))
        assert np.ptp(th) < 1e-9, (e, np.ptp(th))
        assert (t[e] != 0) == (th.min() < 1 - 1e-12)


def test_mrs_leaves_linear_data_alone():
    """Data linear along one axis (the others constant, velocity constant up to
    rounding) stay within the neighbours' means: Theta = 1, even with alpha~ = 0."""
    m = _mrs_mesh(8, 4, 0.0, dim=3)
    x, y, z = m.coords()
    prim = np.stack([1.5 + 0.2 * x, 0.3 + 0 * x, -0.2 + 0 * x, 0.1 + 0 * x, 1.0 + 0.1 * x])
    # periodic wrap breaks linearity at the box edge: check interior elements only
    U = m.from_prim(prim)
    V, t = m.limit(U)
    xc = x.reshape(m.E, -1).mean(axis=1)
    yc = y.reshape(m.E, -1).mean(axis=1)
    zc = z.reshape(m.E, -1).mean(axis=1)
    inner = (np.minimum(xc, 1 - xc) > 0.13) & (np.minimum(yc, 1 - yc) > 0.13) & (np.minimum(zc, 1 - zc) > 0.13)
    assert inner.any() and np.all(t[inner] == 0)
    assert np.array_equal(V[inner], U[inner])


def test_mrs_keeps_smooth_extrema_only_with_alpha():
    """alpha~ > 0 widens the bounds by alpha~ h^{3/2}: on a fine mesh a smooth
    extremum is left alone; with alpha~ = 0 the elements at the extrema are
    clipped (Sec. 3.3.3)."""
    counts = []
    for alpha in (0.0, 50.0):
        m = _mrs_mesh(64, 3, alpha)
        x = m.coords()[0]
        U = m.from_prim(di.smooth_wave_ne(m.coords(), 0.0, k=(1, 1, 1), vel=(0.5, 0.0, 0.0)))
        _, t = m.limit(U)
        counts.append(int((t != 0).sum()))
    assert counts[0] > 0 and counts[1] == 0, counts


def test_mrs_theta_closed_form_for_an_isolated_bump():
    """eq:MRSSol (Sec. 3.3.3) on a density bump in one element of a uniform flow at rest:
    velocity and pressure are constant, so only the density bounds act, the
    neighbours' means lie below the bump's, and Theta = alpha h^{3/2} /
    (rho_max - rho_0), h the element width.  The bump element becomes U0 +
    Theta (U - U0); the others are untouched."""
    K, n, alpha = 8, 4, 0.3
    m = _mrs_mesh(K, n, alpha)
    x = m.coords()[0]
    e0 = 3
    xc, h = (e0 + 0.5) / K, 1.0 / K
    xi = (x - xc) / (0.5 * h)
    bump = np.where(np.abs(x - xc) <= 0.5 * h + 1e-15, 0.2 * (1.0 - xi ** 2), 0.0)
    prim = np.stack([1.0 + bump, np.zeros_like(x), np.zeros_like(x), np.zeros_like(x), np.ones_like(x)])
    U = m.from_prim(prim)
    L, t = m.limit(U)
    S = m.summaries(U)
    rho0 = S[e0, 0, 0]
    theta = alpha * h ** 1.5 / (U[e0, 0].max() - rho0)
    assert 0.2 < theta < 0.8
    assert t[e0] != 0 and np.count_nonzero(t) == 1
    U0 = S[e0, :, 0][:, None]
    assert np.allclose(L[e0], U0 + theta * (U[e0] - U0), rtol=1e-13, atol=1e-14)
    others = np.arange(m.E) != e0
    assert np.array_equal(L[others], U[others])


def test_mrs_needs_newtonian_and_nonnegative_alpha():
    for kw in (dict(system=1, gamma=4.0 / 3.0, mrs_alpha=1.0), dict(system=0, gamma=1.4, mrs_alpha=-1.0)):
        with pytest.raises(Exception):
            oracle.Mesh(oracle.MeshSpec(K=(2, 2, 2), n=3, limiter=3, **kw))
