"""Pins of the oracle's LGL tables (Sec. 3.1, eq:405) against closed forms and
identities that any correct Lobatto basis satisfies."""
import math

import numpy as np
import pytest

import oracle

CLOSED = {
    # Legendre-Gauss-Lobatto nodes and weights in closed form
    2: ([-1.0, 1.0], [1.0, 1.0]),
    3: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    4: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    5: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0], [0.1, 49 / 90, 32 / 45, 49 / 90, 0.1]),
}


@pytest.mark.parametrize("n", sorted(CLOSED))
def test_closed_forms(n):
    x, w = oracle.lgl(n)
    xe, we = CLOSED[n]
    assert np.allclose(x, xe, rtol=0, atol=2e-16)
    assert np.allclose(w, we, rtol=0, atol=4e-16)


@pytest.mark.parametrize("n", range(2, 11))
def test_quadrature_exact_to_degree_2N_minus_1(n):
    x, w = oracle.lgl(n)
    N = n - 1
    assert abs(w.sum() - 2.0) < 1e-14
    for m in range(0, 2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 2e-14, (n, m)
    # degree 2N is NOT integrated exactly by Lobatto quadrature
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-6


@pytest.mark.parametrize("n", range(2, 11))
def test_diffmat_polynomials_and_sbp(n):
    x, w = oracle.lgl(n)
    D = oracle.diffmat(n)
    N = n - 1
    assert np.max(np.abs(D @ np.ones(n))) < 1e-13
    for m in range(1, N + 1):
        err = np.max(np.abs(D @ x ** m - m * x ** (m - 1)))
        assert err < 2e-12 * max(1, N * N), (n, m, err)
    # summation by parts: W D + D^T W = diag(-1, 0, ..., 0, 1)
    W = np.diag(w)
    B = np.zeros((n, n))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.max(np.abs(W @ D + D.T @ W - B)) < 1e-13
    # LGL closed form of the corner entries: D_00 = -N(N+1)/4
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-12 * N * N


@pytest.mark.parametrize("n", range(2, 9))
def test_legendre_vinv_linear_coefficient(n):
    x, w = oracle.lgl(n)
    Vi = oracle.legendre_vinv(n)
    # modal coefficients of a known polynomial c0 + c1 P1 + c2 P2 (degree <= N)
    c = np.zeros(n)
    c[0], c[1] = 0.7, -1.3
    if n > 2:
        c[2] = 0.4
    vals = np.polynomial.legendre.legval(x, c)
    assert np.allclose(Vi @ vals, c, atol=1e-13)
    # P1 coefficient = (3/2) int u xi  (exact by quadrature when N >= 2)
    if n > 2:
        assert np.allclose(Vi[1], 1.5 * w * x, atol=1e-14)
    else:
        assert np.allclose(Vi[1], [-0.5, 0.5], atol=1e-15)
