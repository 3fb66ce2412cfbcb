"""FP64 CPU reference of the learned con2prim starting guess.

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

The network maps three scaled invariants of the SR conserved state to a scaled
log-pressure; con2prim's safeguarded Newton (Sec. 2.1.2) starts from it and alone
decides the result.  Architecture 3 -> 64 -> 64 -> 1 with SiLU activations,
4,481 parameters laid out flat as

    W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3[1]

(W[j][i] maps input i to output j).  Features, with E = tau + D, s = |S|:

    x1 = 2 (log10(tau/D) - lo1) / (hi1 - lo1) - 1
    x2 = 2 s / E - 1                      (s/E in [0, 1) for physical states)
    x3 = 2 (log10 D - lo3) / (hi3 - lo3) - 1

and target y = (log10(p / E) - y_shift) / y_scale.  `scales` holds
(lo1, hi1, lo3, hi3, y_shift, y_scale).  Loss: mean squared error of y.
"""
from __future__ import annotations

import numpy as np

N_HIDDEN = 64
N_PARAMS = 64 * 3 + 64 + 64 * 64 + 64 + 64 + 1  # 4481

DEFAULT_SCALES = (-5.0, 4.0, -9.0, 3.0, -4.5, 4.5)


def unpack(params: np.ndarray) -> dict:
    p = np.asarray(params, dtype=np.float64)
    assert p.size == N_PARAMS
    o = 0
    W1 = p[o:o + 192].reshape(64, 3); o += 192
    b1 = p[o:o + 64]; o += 64
    W2 = p[o:o + 4096].reshape(64, 64); o += 4096
    b2 = p[o:o + 64]; o += 64
    W3 = p[o:o + 64]; o += 64
    b3 = p[o:o + 1]; o += 1
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def pack(d: dict) -> np.ndarray:
    return np.concatenate([d["W1"].ravel(), d["b1"], d["W2"].ravel(), d["b2"], d["W3"], d["b3"]])


OFFSETS = {"W1": 0, "b1": 192, "W2": 256, "b2": 4352, "W3": 4416, "b3": 4480}


def init_params(u: np.ndarray) -> np.ndarray:
    """Initial parameters from uniforms u in [0, 1) (N_PARAMS of them, drawn by the
    caller): weights uniform in +-sqrt(3/fan_in), biases zero."""
    u = np.asarray(u, dtype=np.float64)
    p = np.zeros(N_PARAMS)
    for name, fan, n in (("W1", 3, 192), ("W2", 64, 4096), ("W3", 64, 64)):
        o = OFFSETS[name]
        p[o:o + n] = np.sqrt(3.0 / fan) * (2.0 * u[o:o + n] - 1.0)
    return p


def features(cons: np.ndarray, scales=DEFAULT_SCALES) -> np.ndarray:
    """cons (5, N) -> x (N, 3)."""
    lo1, hi1, lo3, hi3, _, _ = scales
    D, tau = cons[0], cons[4]
    s = np.sqrt(cons[1] ** 2 + cons[2] ** 2 + cons[3] ** 2)
    E = tau + D
    x1 = 2.0 * (np.log10(tau / D) - lo1) / (hi1 - lo1) - 1.0
    x2 = 2.0 * s / E - 1.0
    x3 = 2.0 * (np.log10(D) - lo3) / (hi3 - lo3) - 1.0
    return np.stack([x1, x2, x3], axis=1)


def targets(cons: np.ndarray, p: np.ndarray, scales=DEFAULT_SCALES) -> np.ndarray:
    E = cons[0] + cons[4]
    return (np.log10(p / E) - scales[4]) / scales[5]


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params: np.ndarray, x: np.ndarray):
    """x (N, 3) -> y (N,), and the intermediate values for backward."""
    d = unpack(params)
    z1 = x @ d["W1"].T + d["b1"]
    h1 = silu(z1)
    z2 = h1 @ d["W2"].T + d["b2"]
    h2 = silu(z2)
    y = h2 @ d["W3"] + d["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray):
    """Mean squared error over the batch and its gradient (flat, N_PARAMS)."""
    d = unpack(params)
    y, (x, z1, h1, z2, h2) = forward(params, x)
    B = x.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, d["W3"]) * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ d["W2"]) * dsilu(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) with bias correction; returns new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def guess(params: np.ndarray, cons: np.ndarray, gamma: float, scales=DEFAULT_SCALES) -> np.ndarray:
    """Pressure guess E 10^(y y_scale + y_shift), clamped into con2prim's bracket
    [max(0, s - E), (gamma - 1) tau]."""
    y, _ = forward(params, features(cons, scales))
    D, tau = cons[0], cons[4]
    s = np.sqrt(cons[1] ** 2 + cons[2] ** 2 + cons[3] ** 2)
    E = tau + D
    p = E * 10.0 ** (y * scales[5] + scales[4])
    return np.clip(p, np.maximum(0.0, s - E), (gamma - 1.0) * tau)
