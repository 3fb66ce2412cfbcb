"""Pins of the FP64 MLP reference of the learned con2prim guess: gradients
against central finite differences, the Adam update against its definition on
a quadratic, and the feature map against its defining formulas."""
import numpy as np
import pytest

import dg_inputs as di
import oracle
from oracle import mlp


def _batch(n=64, seed=3):
    g = 4.0 / 3.0
    prim = di.c2p_samples(seed, n, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    return cons, prim[4]


def test_parameter_count_and_layout():
    assert mlp.N_PARAMS == 4481
    p = np.arange(mlp.N_PARAMS, dtype=float)
    d = mlp.unpack(p)
    assert d["W1"].shape == (64, 3) and d["W2"].shape == (64, 64) and d["b3"].shape == (1,)
    assert np.array_equal(mlp.pack(d), p)


def test_gradient_matches_central_differences():
    cons, p = _batch()
    x, t = mlp.features(cons), mlp.targets(cons, p)
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng.random(mlp.N_PARAMS))
    params[mlp.OFFSETS["b1"]:mlp.OFFSETS["b1"] + 64] = 0.1 * rng.standard_normal(64)
    loss, g = mlp.loss_and_grad(params, x, t)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [mlp.N_PARAMS - 1, 0, 200]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        lp, _ = mlp.loss_and_grad(params + e, x, t)
        lm, _ = mlp.loss_and_grad(params - e, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_adam_on_a_quadratic():
    # Adam's first step moves every coordinate by lr (bias-corrected m/sqrt(v) = sign(g))
    p = np.array([1.0, -2.0, 3.0])
    g = 2.0 * p
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(p), rtol=0, atol=1e-10)
    for k in range(2, 400):
        p1, m, v = mlp.adam_step(p1, 2.0 * p1, m, v, k, lr=0.05)
    assert np.abs(p1).max() < 0.1


def test_features_and_guess_bracket():
    cons, p = _batch(200)
    x = mlp.features(cons)
    D, tau = cons[0], cons[4]
    s = np.sqrt((cons[1:4] ** 2).sum(axis=0))
    assert np.allclose((x[:, 1] + 1) / 2, s / (tau + D))
    assert np.all(np.abs(x) <= 1.0)
    params = mlp.init_params(np.random.default_rng(1).random(mlp.N_PARAMS))
    pg = mlp.guess(params, cons, 4.0 / 3.0)
    assert np.all(pg >= np.maximum(0, s - tau - D)) and np.all(pg <= (4 / 3 - 1) * tau)


def test_silu_identities():
    """SiLU z sigma(z): silu(0) = 0, silu(z) - silu(-z) = z, silu(z) -> z for large
    z, and its derivative matches central differences."""
    z = np.linspace(-8.0, 8.0, 161)
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.silu(z) - mlp.silu(-z), z, rtol=0, atol=1e-14)
    assert abs(mlp.silu(np.array([40.0]))[0] - 40.0) < 1e-14
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.dsilu(z), fd, rtol=0, atol=1e-8)


def test_planted_errors_in_the_mlp_are_caught(monkeypatch):
    """A wrong SiLU derivative in backward, and a SiLU with the wrong sign in its
    exponent, are rejected by the pins above: planted in the oracle on the CPU."""
    good = mlp.dsilu

    def bad_dsilu(z):
        s = 1.0 / (1.0 + np.exp(-z))
        return s * (1.0 + z * s)

    monkeypatch.setattr(mlp, "dsilu", bad_dsilu)
    with pytest.raises(AssertionError):
        test_gradient_matches_central_differences()
    monkeypatch.setattr(mlp, "dsilu", good)
    monkeypatch.setattr(mlp, "silu", lambda z: z / (1.0 + np.exp(z)))
    with pytest.raises(AssertionError):
        test_silu_identities()
