"""Analytic outer boundaries on the GPU (Sec. 3.4) with the isentropic vortex
(eq:isen_vortex, tab:IsenVortexConvergence).  Interior elements give the oracle's
bits; elements on an analytic face agree to rounding (CUDA's exp and pow against
libm's in the exterior state); steps, the mesh time and the paper's error table
follow, for FP64 and mixed precision."""
import math

import numpy as np
import pytest

import dg_inputs as di
import oracle

pytestmark = pytest.mark.gpu

V = di.VORTEX


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as p
    from paper_1609_00098_gb300 import build as b
    b.build()
    return p


def _gpu(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _kw(K, n, flux=0, bc=(1, 1, 1), x0=V["x0"], y0=V["y0"]):
    return dict(system=0, K=K, n=n, flux=flux, limiter=0, gamma=V["gamma"], lo=(0, 0, 0), hi=(10, 10, 1), bc=bc,
                exact=1, exact_par=(V["beta"], x0, y0, *V["vel"]))


def _pair(pkg, precision=0, **kw):
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    gm = pkg.Mesh(precision=precision, **kw)
    return om, gm


@pytest.mark.parametrize("flux", [0, 1, 2])
def test_vortex_rhs_fp64(pkg, flux):
    """RHS at t = 0.3 with analytic x and y faces: bitwise on elements away from
    them, to 1e-13 (relative to the variable's largest RHS) on the rest."""
    om, gm = _pair(pkg, **_kw((5, 4, 2), 3, flux=flux, bc=(1, 1, 0)))
    U = om.from_prim(di.isentropic_vortex(om.coords(), 0.0))
    om.t = 0.3
    gm.t = 0.3
    Ro = om.rhs(U)
    Rg = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    ec = np.arange(om.E)
    ex, ey = ec % 5, (ec // 5) % 4
    inner = (ex > 0) & (ex < 4) & (ey > 0) & (ey < 3)
    assert np.array_equal(Rg[inner], Ro[inner])
    sc = np.abs(Ro).max(axis=(0, 2))
    assert np.all(np.abs(Rg - Ro).max(axis=(0, 2)) <= 1e-13 * sc)
    om.t = 0.0
    assert not np.array_equal(om.rhs(U)[~inner], Ro[~inner])  # the exterior state follows the time


def test_vortex_steps_fp64_and_time(pkg):
    """Twenty fixed-dt SSP-RK3 steps (exterior states at t, t + dt, t + dt/2) of a
    vortex leaving through the hi corner: within 1e-12 of the oracle, and the mesh
    time equals the oracle's."""
    om, gm = _pair(pkg, **_kw((8, 8, 1), 4, x0=8.5, y0=8.5))
    U = om.from_prim(di.isentropic_vortex(om.coords(), 0.0, x0=8.5, y0=8.5))
    Ug = _gpu(U)
    dt = 0.02
    for _ in range(20):
        U = om.rk3_step(U, dt)
        gm.rk3_step(Ug, dt=dt)
    assert gm.sync_status() == 0
    assert gm.t == om.t
    sc = np.abs(U).max(axis=(0, 2))
    assert np.all(np.abs(Ug.cpu().numpy() - U).max(axis=(0, 2)) <= 1e-12 * sc)


def test_vortex_ab3_and_cfl_time(pkg):
    """Adams-Bashforth steps advance the mesh time like SSP-RK3; CFL steps advance
    it by the device dt."""
    import torch
    om, gm = _pair(pkg, **_kw((4, 4, 1), 3))
    U = om.from_prim(di.isentropic_vortex(om.coords(), 0.0))
    dt = 0.01
    Uo = om.ab3_run(U, 5, dt)
    Ug = _gpu(U)
    for _ in range(5):
        gm.ab3_step(Ug, dt)
    assert abs(gm.t - om.t) < 1e-15 and abs(om.t - 0.05) < 1e-15
    sc = np.abs(Uo).max(axis=(0, 2))
    assert np.all(np.abs(Ug.cpu().numpy() - Uo).max(axis=(0, 2)) <= 1e-12 * sc)
    gm.t = 0.0
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    tot = 0.0
    for _ in range(3):
        gm.rk3_step(Ug, cfl=0.2, dt_used=d)
        tot += float(d.item())
    assert gm.t == pytest.approx(tot, rel=1e-15)


def _gpu_vortex_error(pkg, nc, K, precision, T=2.0, cfl=0.2):
    import torch
    kw = _kw((K, K, 1), nc)
    gm = pkg.Mesh(precision=precision, **kw)
    xyz = gm.coords()
    U = gm.from_prim(torch.from_numpy(di.isentropic_vortex(xyz.cpu().numpy(), 0.0)).cuda())
    om = oracle.Mesh(oracle.MeshSpec(**kw))   # norms only
    steps = int(math.ceil(T / om.cfl_dt(om.from_prim(di.isentropic_vortex(om.coords(), 0.0)), cfl)))
    dt = T / steps
    for _ in range(steps):
        gm.rk3_step(U, dt=dt)
    assert gm.sync_status() == 0
    assert abs(gm.t - T) < 1e-12
    Uex = om.from_prim(di.isentropic_vortex(om.coords(), T))
    Uh = U.cpu().numpy()
    return om.norms(Uh, Uex)[0].sum(), steps, dt, Uh, om


def test_vortex_table_entry_fp64_and_mixed(pkg):
    """tab:IsenVortexConvergence at N_C = 5, K = 16 (printed 7.98e-3): the FP64 path
    gives the oracle's error to 1e-9; the mixed state is within 1e-6 relative L2 of
    the FP64 one (FP32 rounding of the RHS, about 1e-7 of the state, moves the L1
    error by ~1e-5: a floor the finer table entries would reach)."""
    e64, steps, dt, U64, om64 = _gpu_vortex_error(pkg, 5, 16, 0)
    om = oracle.Mesh(oracle.MeshSpec(**_kw((16, 16, 1), 5)))
    xyz = om.coords()
    U = om.from_prim(di.isentropic_vortex(xyz, 0.0))
    for _ in range(steps):
        U = om.rk3_step(U, dt)
    eo = om.norms(U, om.from_prim(di.isentropic_vortex(xyz, 2.0)))[0].sum()
    assert abs(e64 / eo - 1) < 1e-9, (e64, eo)
    assert abs(e64 / 7.98e-3 - 1) < 0.15
    emx, _, _, Umx, _ = _gpu_vortex_error(pkg, 5, 16, 1)
    assert abs(emx / e64 - 1) < 1e-2, (emx, e64)
    _, d = om64.norms(Umx, U64)
    _, ref = om64.norms(U64, np.zeros_like(U64))
    rel = d / np.maximum(ref, 1e-2 * ref.max())
    assert np.all(rel <= 1e-6), rel


TABLE = {4: (6.70e-3, 3.44e-4, 2.15e-5), 5: (3.13e-4, 1.44e-5, 6.94e-7)}  # K = 32, 64, 128


@pytest.mark.parametrize("nc", [4, 5])
def test_vortex_table_full_size_fp64(pkg, nc):
    """Table rows N_C = 4, 5 at K = 32, 64, 128 (beyond the oracle's reach) on the
    FP64 path: each error within a factor 1.4 of the printed one (the oracle sits
    within 15 % on coarse meshes; the gap grows to 1.2-1.35 here and does not close
    at the paper's dt = 1e-4), and the local convergence orders within 0.3 of the
    printed orders."""
    e = [_gpu_vortex_error(pkg, nc, K, 0)[0] for K in (32, 64, 128)]
    ref = TABLE[nc]
    for a, b in zip(e, ref):
        assert 1 / 1.4 < a / b < 1.4, (e, ref)
    for k in range(2):
        assert abs(math.log2(e[k] / e[k + 1]) - math.log2(ref[k] / ref[k + 1])) < 0.3, (e, ref)


def test_analytic_boundaries_rejected(pkg):
    for kw in (dict(limiter=1), dict(system=1, flux=1, gamma=4.0 / 3.0), dict(exact=0)):
        args = dict(_kw((2, 2, 1), 3), **kw)
        with pytest.raises(pkg.abi.DGError):
            pkg.Mesh(precision=1, **args)
    m = pkg.Mesh(precision=1, **_kw((2, 2, 1), 3))
    with pytest.raises(pkg.abi.DGError):
        pkg.abi.dg_ensemble_create([m.h], [m.state()])
