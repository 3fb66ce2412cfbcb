"""The seeded input generators (`dg_inputs`), which both the oracle and the CUDA
path take their inputs from: the counter-based generator against its published
definition, and each problem's initial data against what defines it
(tab:Riemann_Problems; the blast and Kelvin-Helmholtz recipes; the con2prim and
ensemble sampling ranges)."""
import os

import numpy as np
import pytest

import dg_inputs as di

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA64 = 0x9E3779B97F4A7C15  # SplitMix64's state increment


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) seeded with 0 emits these five
    values first; its k-th output is the finaliser of k times the increment."""
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                0x1B39896A51A8749B]
    counters = np.array([(k * GAMMA64) % 2**64 for k in range(5)], dtype=np.uint64)
    assert [int(v) for v in di.splitmix64(counters)] == expected


def test_uniform_counter_layout_and_range():
    idx = np.arange(100_000)
    u = di.uniform(3, 1, idx)
    assert u.dtype == np.float64 and u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005
    # the top 53 bits of the generator at key (seed << 44) ^ (stream << 36) ^ index
    key = (np.uint64(3) << np.uint64(44)) ^ (np.uint64(1) << np.uint64(36)) ^ idx[:8].astype(np.uint64)
    top = (di.splitmix64(key) >> np.uint64(11)).astype(np.float64)
    assert np.array_equal(u[:8], top / 2.0**53)
    # reproducible; other seeds and streams give other numbers
    assert np.array_equal(u, di.uniform(3, 1, idx))
    assert not np.any(u[:1000] == di.uniform(4, 1, idx[:1000]))
    assert not np.any(u[:1000] == di.uniform(3, 2, idx[:1000]))


def _grid(lo, hi, m=24):
    x = np.linspace(lo, hi, m)
    return np.stack(np.meshgrid(x, x, x, indexing="ij"))


def test_riemann_problems_match_the_printed_table():
    rows = {}
    with open(os.path.join(GOLDEN, "riemann_problems.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = [float(v) for v in vals]
    assert set(rows) == set(di.RIEMANN)
    for name, vals in rows.items():
        np.testing.assert_allclose(di.RIEMANN[name], vals, rtol=1e-10, atol=0.0)
        rl, ul, pl, rr, ur, pr, _g, xd = di.RIEMANN[name]
        x = np.linspace(-1.0, 1.0, 41)
        xyz = np.stack([x, np.zeros_like(x), np.zeros_like(x)])
        w = di.riemann_1d(xyz, name)
        left = x <= xd
        assert np.all(w[0][left] == rl) and np.all(w[0][~left] == rr)
        assert np.all(w[1][left] == ul) and np.all(w[1][~left] == ur)
        assert np.all(w[4][left] == pl) and np.all(w[4][~left] == pr)
        assert np.all(w[2] == 0.0) and np.all(w[3] == 0.0)


def test_kelvin_helmholtz_recipe():
    """Shear layer on [-0.5, 0.5]^3: rho = 2, v_x = +0.5 in |y| < 0.25, else rho = 1,
    v_x = -0.5; v_y = 0.01 (2u - 1) per node; v_z = 0; p = 2.5."""
    xyz = _grid(-0.5, 0.5)
    w = di.kh_ne(xyz, seed=1)
    inside = np.abs(xyz[1]) < 0.25
    assert np.all(w[0][inside] == 2.0) and np.all(w[0][~inside] == 1.0)
    assert np.all(w[1][inside] == 0.5) and np.all(w[1][~inside] == -0.5)
    assert np.all(np.abs(w[2]) <= 0.01) and abs(w[2].mean()) < 5e-4 and w[2].std() > 0.005
    assert np.all(w[3] == 0.0) and np.all(w[4] == 2.5)
    assert not np.array_equal(w[2], di.kh_ne(xyz, seed=2)[2])
    assert np.array_equal(w, di.kh_ne(xyz, seed=1))


def test_blast_recipe():
    """Sphere of radius 0.3 about (0.5, 0.5, 0.5): rho = 10, p = 13.33 inside, rho = 1,
    p = 1e-6 outside, at rest, the density times 1 + 0.01 (2u - 1) per node."""
    xyz = _grid(0.0, 1.0)
    w = di.blast_sr(xyz, seed=1)
    r2 = ((xyz - 0.5) ** 2).sum(axis=0)
    inside = r2 < 0.09
    assert inside.any() and (~inside).any()
    ratio = w[0] / np.where(inside, 10.0, 1.0)
    assert np.all(np.abs(ratio - 1.0) <= 0.01 + 1e-15) and ratio.std() > 0.004
    assert np.all(w[4][inside] == 13.33) and np.all(w[4][~inside] == 1e-6)
    assert np.all(w[1:4] == 0.0)


def test_con2prim_sample_ranges():
    """rho log-uniform in [1e-8, 10], W uniform in [1, 10], eps log-uniform in
    [1e-6, 1e2], p = (gamma - 1) rho eps."""
    gamma = 4.0 / 3.0
    w = di.c2p_samples(seed=3, count=200_000, gamma=gamma)
    rho, v, p = w[0], w[1:4], w[4]
    assert rho.min() >= 1e-8 and rho.max() < 10.0
    lr = np.log10(rho)
    assert abs(lr.mean() - (-3.5)) < 0.05
    v2 = (v * v).sum(axis=0)
    W = 1.0 / np.sqrt(1.0 - v2)
    assert W.min() >= 1.0 - 1e-12 and W.max() <= 10.0 + 1e-9 and abs(W.mean() - 5.5) < 0.05
    eps = p / ((gamma - 1.0) * rho)
    assert eps.min() >= 1e-6 * (1 - 1e-12) and eps.max() <= 1e2 * (1 + 1e-12)
    # directions uniform on the sphere: each velocity component's mean is zero
    assert np.all(np.abs((v / np.sqrt(v2)).mean(axis=1)) < 0.01)
    # a slice of the stream equals the same states drawn from its start index
    np.testing.assert_array_equal(di.c2p_samples(3, 10, start=100, gamma=gamma), w[:, 100:110])


def test_ensemble_recipe_ranges():
    rec = di.ensemble_recipe(5)
    assert len(rec) == 256 and rec == di.ensemble_recipe(5)
    systems = [s for s, _, _ in rec]
    assert set(systems) == {0, 1} and 96 < sum(systems) < 160
    assert {K for _, K, _ in rec} <= set(range(2, 17)) and {n for _, _, n in rec} == set(range(3, 9))
    assert min(K for _, K, _ in rec) == 2 and max(K for _, K, _ in rec) == 16


@pytest.mark.parametrize("k", [(1, 1, 1), (2, 1, 2)])
def test_smooth_wave_is_advected(k):
    """rho(x, t) = rho(x - v t, 0): the exact solution moves with the uniform flow."""
    xyz = _grid(0.0, 1.0, 9)
    vel = (1.0, 0.5, 0.25)
    t = 0.3
    shifted = xyz - np.array(vel).reshape(3, 1, 1, 1) * t
    np.testing.assert_allclose(di.smooth_wave_ne(xyz, t=t, k=k, vel=vel)[0],
                               di.smooth_wave_ne(shifted, t=0.0, k=k, vel=vel)[0], rtol=0, atol=1e-13)
