"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds NO arithmetic of the DG method: it only draws counter-based
random numbers and evaluates the problems' primitive fields (rho, v, p) at node
coordinates the caller supplies.  Node coordinates (LGL nodes) and the
primitive->conserved map belong to each side and are computed there.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) applied to the counter
``key = (seed << 44) ^ (stream << 36) ^ index``; the top 53 bits give u in [0, 1).

Problems (initial data of the paper's tests, Sec. 6, and of the workloads this
library is measured on):
  * ``smooth_wave_ne``: advected density wave, Newtonian Euler, p = 1;
  * ``smooth_flow_re``: eq:smooth_flow_re (Sec. 6.2.2), relativistic, p = 1;
  * ``blast_sr``: spherical relativistic blast, rho=10, p=13.33 for r<0.3 else
    rho=1, p=1e-6, v=0, with 1% seeded density noise;
  * ``kh_ne``: Kelvin-Helmholtz shear layer, Newtonian;
  * ``isentropic_vortex``: eq:isen_vortex (Sec. 6.2.1), Newtonian, at any t;
  * ``riemann_1d``: the Riemann problems of tab:Riemann_Problems (Sec. 6.1);
  * ``c2p_samples``: random primitive states for con2prim;
  * ``ensemble_recipe``: the (system, K, n) list of a ragged ensemble.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of a uint64 counter array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """u in [0, 1) for each counter ``index`` (array of non-negative ints < 2^36)."""
    idx = np.asarray(index, dtype=np.uint64)
    key = (np.uint64(seed) << np.uint64(44)) ^ (np.uint64(stream) << np.uint64(36)) ^ idx
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# random streams
STREAM_NOISE = 1
STREAM_WAVE = 2
STREAM_C2P = 3
STREAM_ENSEMBLE = 4


def _prim(rho, vx, vy, vz, p) -> np.ndarray:
    n = np.broadcast(rho, vx, vy, vz, p).shape
    out = np.empty((5,) + n)
    out[0], out[1], out[2], out[3], out[4] = rho, vx, vy, vz, p
    return out


def wave_numbers(seed: int) -> tuple[int, int, int]:
    """Integer wave numbers k in {1, 2} per axis drawn from the seed."""
    u = uniform(seed, STREAM_WAVE, np.arange(3))
    return tuple(int(1 + math.floor(2.0 * ui)) for ui in u)


def smooth_wave_ne(xyz: np.ndarray, t: float = 0.0, k=(1, 1, 1), amp: float = 0.2,
                   vel=(1.0, 0.5, 0.25), p: float = 1.0) -> np.ndarray:
    """rho = 1 + amp sin(2 pi k.(x - v t)), uniform v and p (exact solution at t)."""
    x, y, z = xyz
    ph = 2.0 * math.pi * (k[0] * (x - vel[0] * t) + k[1] * (y - vel[1] * t) + k[2] * (z - vel[2] * t))
    rho = 1.0 + amp * np.sin(ph)
    return _prim(rho, vel[0], vel[1], vel[2], p)


def smooth_flow_re(xyz: np.ndarray, t: float = 0.0, amp: float = 0.2, k: float = 2 * math.pi,
                   vel=(0.2, 0.2, 0.2), gamma: float = 5.0 / 3.0, dim: int = 3) -> np.ndarray:
    """eq:smooth_flow_re: rho = 1 + A sin(u), eps = 1/((gamma-1) rho) so p = 1,
    u = k [sum_a x_a - (sum_a v_a) t] over the active axes."""
    s = np.zeros_like(xyz[0])
    vs = 0.0
    for a in range(dim):
        s = s + xyz[a]
        vs += vel[a]
    u = k * (s - vs * t)
    rho = 1.0 + amp * np.sin(u)
    v = [vel[a] if a < dim else 0.0 for a in range(3)]
    return _prim(rho, v[0], v[1], v[2], 1.0)


def blast_sr(xyz: np.ndarray, seed: int, center=(0.5, 0.5, 0.5), radius: float = 0.3,
             rho_in: float = 10.0, p_in: float = 13.33, rho_out: float = 1.0,
             p_out: float = 1e-6, noise: float = 0.01) -> np.ndarray:
    """Relativistic blast: rho_in, p_in inside r < radius, else rho_out, p_out,
    v = 0, density times (1 + noise (2u - 1)) per node (u from the node index)."""
    x, y, z = xyz
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
    inside = r2 < radius * radius
    u = uniform(seed, STREAM_NOISE, np.arange(x.size)).reshape(x.shape)
    rho = np.where(inside, rho_in, rho_out) * (1.0 + noise * (2.0 * u - 1.0))
    p = np.where(inside, p_in, p_out)
    return _prim(rho, 0.0, 0.0, 0.0, p)


def kh_ne(xyz: np.ndarray, seed: int, p: float = 2.5, amp: float = 0.01) -> np.ndarray:
    """Kelvin-Helmholtz shear layer on [-0.5, 0.5]^3: rho = 2, vx = +0.5 for
    |y| < 0.25, else rho = 1, vx = -0.5; vy = amp (2u - 1) per node; p uniform."""
    x, y, z = xyz
    inside = np.abs(y) < 0.25
    rho = np.where(inside, 2.0, 1.0)
    vx = np.where(inside, 0.5, -0.5)
    u = uniform(seed, STREAM_NOISE, np.arange(x.size)).reshape(x.shape)
    vy = amp * (2.0 * u - 1.0)
    return _prim(rho, vx, vy, 0.0, p)


VORTEX = dict(beta=5.0, x0=4.0, y0=4.0, vel=(1.0, 1.0, 0.0), gamma=1.4)  # tab:IsenVortexConvergence


def isentropic_vortex(xyz: np.ndarray, t: float = 0.0, beta: float = 5.0, x0: float = 4.0, y0: float = 4.0,
                      vel=(1.0, 1.0, 0.0), gamma: float = 1.4) -> np.ndarray:
    """eq:isen_vortex at time t: with xt = x - x0 - U t, yt = y - y0 - V t and
    r^2 = xt^2 + yt^2, rho = (1 - (gamma-1) beta^2 e^(1-r^2) / (8 gamma pi^2))^(1/(gamma-1)),
    v = (U - yt f, V + xt f, W) with f = beta e^((1-r^2)/2) / (2 pi), p = rho^gamma."""
    x, y, _ = xyz
    xt = x - x0 - vel[0] * t
    yt = y - y0 - vel[1] * t
    r2 = xt * xt + yt * yt
    rho = (1.0 - (gamma - 1.0) * beta * beta * np.exp(1.0 - r2) / (8.0 * gamma * math.pi ** 2)) ** (1.0 / (gamma - 1.0))
    f = beta * np.exp(0.5 * (1.0 - r2)) / (2.0 * math.pi)
    return _prim(rho, vel[0] - yt * f, vel[1] + xt * f, vel[2] + 0.0 * x, rho ** gamma)


RIEMANN = {
    # name: (rho_L, u_L, p_L, rho_R, u_R, p_R, gamma, x_d)  -- tab:Riemann_Problems
    "sod": (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, 0.0),
    "st1": (10.0, 0.0, 13.33, 1.0, 0.0, 1e-8, 5.0 / 3.0, 0.5),
    "st2": (1.0, 0.0, 1000.0, 1.0, 0.0, 1e-2, 5.0 / 3.0, 0.5),
}


def riemann_1d(xyz: np.ndarray, name: str) -> np.ndarray:
    rl, ul, pl, rr, ur, pr, _g, xd = RIEMANN[name]
    x = xyz[0]
    left = x <= xd
    return _prim(np.where(left, rl, rr), np.where(left, ul, ur), 0.0, 0.0, np.where(left, pl, pr))


def c2p_samples(seed: int, count: int, start: int = 0, gamma: float = 4.0 / 3.0) -> np.ndarray:
    """Random primitive states: rho log-uniform [1e-8, 10], Lorentz factor W
    uniform [1, 10] on a uniformly random direction, eps log-uniform [1e-6, 1e2],
    p = (gamma - 1) rho eps.  Returns (5, count) rows rho, vx, vy, vz, p."""
    base = (np.arange(count, dtype=np.int64) + start) * 5
    u0 = uniform(seed, STREAM_C2P, base + 0)
    u1 = uniform(seed, STREAM_C2P, base + 1)
    u2 = uniform(seed, STREAM_C2P, base + 2)
    u3 = uniform(seed, STREAM_C2P, base + 3)
    u4 = uniform(seed, STREAM_C2P, base + 4)
    rho = 10.0 ** (-8.0 + 9.0 * u0)
    W = 1.0 + 9.0 * u1
    ct = 2.0 * u2 - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * math.pi * u3
    eps = 10.0 ** (-6.0 + 8.0 * u4)
    vmag = np.sqrt(1.0 - 1.0 / (W * W))
    p = (gamma - 1.0) * rho * eps
    return _prim(rho, vmag * st * np.cos(ph), vmag * st * np.sin(ph), vmag * ct, p)


def ensemble_recipe(seed: int, count: int = 256, kmin: int = 2, kmax: int = 16,
                    nmin: int = 3, nmax: int = 8):
    """(system, K, n) per mesh: system 0/1 with probability 1/2, K uniform in
    [kmin, kmax], n uniform in [nmin, nmax]."""
    out = []
    for m in range(count):
        u = uniform(seed, STREAM_ENSEMBLE, np.arange(3) + 3 * m)
        system = int(u[0] >= 0.5)
        K = kmin + min(int(u[1] * (kmax - kmin + 1)), kmax - kmin)
        n = nmin + min(int(u[2] * (nmax - nmin + 1)), nmax - nmin)
        out.append((system, K, n))
    return out
