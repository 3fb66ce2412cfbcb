"""GPU vs oracle parity of the FP64 CUDA path, element by element, through the
C ABI.  Tolerance: relative max-norm per variable <= 1e-12 (the bar for the FP64
path), scale = max |oracle| of that variable."""
import math

import numpy as np
import pytest

import dg_inputs as di
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as p
    from paper_1609_00098_gb300 import build as b
    b.build()
    return p


def _rel(got, ref, axis=(0, 2)):
    scale = np.maximum(np.abs(ref).max(axis=axis), 1e-300)
    return np.abs(got - ref).max(axis=axis) / scale


def _pair(pkg, system=0, K=(4, 4, 4), n=4, flux=0, limiter=0, gamma=None, lo=(0, 0, 0), hi=(1, 1, 1),
          **kw):
    gamma = gamma or (1.4 if system == 0 else 4.0 / 3.0)
    spec = oracle.MeshSpec(system=system, K=K, n=n, flux=flux, limiter=limiter, gamma=gamma, lo=lo, hi=hi, **kw)
    om = oracle.Mesh(spec)
    gm = pkg.Mesh(system=system, K=K, n=n, flux=flux, limiter=limiter, gamma=gamma, lo=lo, hi=hi, **kw)
    return om, gm


def _init(om, kind, seed=1):
    xyz = om.coords()
    if kind == "wave":
        return om.from_prim(di.smooth_wave_ne(xyz, k=di.wave_numbers(seed)))
    if kind == "blast":
        return om.from_prim(di.blast_sr(xyz, seed=seed))
    if kind == "kh":
        return om.from_prim(di.kh_ne(xyz, seed=seed))
    if kind == "re_smooth":
        return om.from_prim(di.smooth_flow_re(xyz, gamma=om.spec.gamma))
    raise ValueError(kind)


def _gpu(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_tables_coords_prim2con(pkg):
    import torch
    om, gm = _pair(pkg, system=1, K=(3, 2, 5), n=5, lo=(-1, 0, 2), hi=(1, 0.5, 3))
    xo = om.coords()
    xg = gm.coords().cpu().numpy()
    assert np.abs(xg - xo).max() <= 4e-16 * np.abs(xo).max()
    prim = di.blast_sr(xo, seed=3)
    Ug = gm.from_prim(_gpu(prim)).cpu().numpy()
    Uo = om.from_prim(prim)
    assert _rel(Ug, Uo).max() <= 1e-15


@pytest.mark.parametrize("system,flux,kind,n", [(0, 0, "wave", 4), (0, 1, "kh", 3), (1, 1, "blast", 5),
                                                (1, 0, "re_smooth", 2), (0, 1, "wave", 8), (1, 1, "blast", 7)])
def test_rhs_parity(pkg, system, flux, kind, n):
    lo, hi = ((-0.5,) * 3, (0.5,) * 3) if kind == "kh" else ((0, 0, 0), (1, 1, 1))
    om, gm = _pair(pkg, system=system, K=(3, 4, 2), n=n, flux=flux, lo=lo, hi=hi)
    U = _init(om, kind)
    Ro = om.rhs(U)
    Rg = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    assert _rel(Rg, Ro).max() <= TOL, _rel(Rg, Ro)


def test_primitives_and_dt_parity(pkg):
    import torch
    om, gm = _pair(pkg, system=1, K=(4, 4, 4), n=5, flux=1)
    U = _init(om, "blast")
    Pg = gm.primitives(_gpu(U)).cpu().numpy()
    Po = om.primitives(U)
    assert _rel(Pg, Po).max() <= TOL
    dtg = gm.cfl_dt(_gpu(U), 0.2).item()
    dto = om.cfl_dt(U, 0.2)
    assert abs(dtg - dto) <= 4e-16 * dto


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_limiter_parity(pkg, n):
    import torch
    om, gm = _pair(pkg, system=1, K=(4, 3, 3), n=n, flux=1, limiter=1)
    U = _init(om, "blast", seed=2)
    So = om.summaries(U)
    Sg = gm.summaries(_gpu(U)).cpu().numpy()
    assert _rel(Sg, So, axis=(0,)).max() <= 1e-13
    Lo, to = om.limit(U)
    t = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    Ug = _gpu(U)
    gm.limit(Ug, t)
    assert np.array_equal(t.cpu().numpy(), to)
    assert _rel(Ug.cpu().numpy(), Lo).max() <= TOL


def test_config1_ten_steps(pkg):
    """Newtonian smooth wave, K=4, n=4, Rusanov, CFL 0.2, 10 steps, no limiter:
    GPU (dt from the device CFL reduction) vs oracle, and both vs the exact solution."""
    import torch
    om, gm = _pair(pkg, system=0, K=(4, 4, 4), n=4, flux=0)
    k = di.wave_numbers(1)
    U0 = om.from_prim(di.smooth_wave_ne(om.coords(), k=k))
    Uo = U0.copy()
    t = 0.0
    for _ in range(10):
        h = om.cfl_dt(Uo, 0.2)
        Uo = om.rk3_step(Uo, h)
        t += h
    Ug = _gpu(U0)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    tg = 0.0
    for _ in range(10):
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt)
        tg += dt.item()
    assert gm.sync_status() == 0
    assert abs(tg - t) <= 1e-14 * t
    assert _rel(Ug.cpu().numpy(), Uo).max() <= TOL
    Uex = om.from_prim(di.smooth_wave_ne(om.coords(), t, k=k))
    eo = om.norms(Uo, Uex)[1]
    eg = om.norms(Ug.cpu().numpy(), Uex)[1]
    assert np.allclose(eg, eo, rtol=1e-9)


@pytest.mark.parametrize("limiter", [1, 2])
def test_blast_steps_with_limiter(pkg, limiter):
    """SR blast, HLL, limiter after every stage, fix: 10 CFL steps, troubled flags of
    each step's last stage compared first, then the state."""
    import torch
    om, gm = _pair(pkg, system=1, K=(5, 4, 4), n=5, flux=1, limiter=limiter)
    U = _init(om, "blast")
    Ug = _gpu(U)
    Uo = U.copy()
    tg = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    for step in range(10):
        h = om.cfl_dt(Uo, 0.2)
        to = np.zeros(om.E, dtype=np.uint8)
        Uo = om.rk3_step(Uo, h, to)
        gm.rk3_step(Ug, dt=h, troubled=tg)
        assert np.array_equal(tg.cpu().numpy(), to), f"troubled flags differ at step {step}"
    assert gm.sync_status() == 0
    assert _rel(Ug.cpu().numpy(), Uo).max() <= TOL, _rel(Ug.cpu().numpy(), Uo)


def test_con2prim_parity(pkg):
    import torch
    g = 4.0 / 3.0
    prim = di.c2p_samples(9, 200000, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    po, ito, sto = oracle.con2prim(g, cons)
    N = cons.shape[1]
    pg = torch.empty((5, N), dtype=torch.float64, device="cuda")
    it = torch.empty(N, dtype=torch.int32, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    pkg.abi.dg_con2prim(N, g, _gpu(cons), pg, None, it, st)
    pg = pg.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    rel = np.abs(pg - po) / np.maximum(np.abs(po), 1e-300)
    assert rel[[0, 4]].max() <= TOL
    vmag = np.sqrt((po[1:4] ** 2).sum(axis=0)) + 1e-300
    assert (np.abs(pg[1:4] - po[1:4]) / vmag).max() <= TOL
    # same IEEE operations in the same order: identical primitives and iteration counts
    assert np.array_equal(pg, po)
    assert np.array_equal(it.cpu().numpy(), ito)
    # a guess at the root converges in one or two steps where f is well resolved
    out = torch.empty((5, N), dtype=torch.float64, device="cuda")
    pkg.abi.dg_con2prim(N, g, _gpu(cons), out, _gpu(po[4]), it, st)
    its = it.cpu().numpy()
    kappa = cons[4] / (po[4] / (g - 1.0))
    assert np.all(its[kappa < 10] <= 3) and np.median(its) <= 2 and its.mean() < ito.mean()
    assert np.all(np.abs(out.cpu().numpy()[4] - po[4]) <= 4e-15 * (1.0 + kappa) * po[4])


def test_edge_cases_shapes(pkg):
    """Self-periodic K=1 axes, ragged K, anisotropic boxes, both extreme n."""
    for K, n, system in [((1, 1, 1), 2, 0),
                             ((1, 3, 1), 8, 1),
                             ((7, 1, 2), 3, 1)]:
        om, gm = _pair(pkg, system=system, K=K, n=n, flux=1, limiter=1, lo=(0, -2, 0), hi=(1, 1, 0.25))
        U = _init(om, "wave" if system == 0 else "blast")
        Uo = om.rk3_step(U, 0.3 * om.cfl_dt(U, 0.2))
        Ug = _gpu(U)
        gm.rk3_step(Ug, dt=0.3 * om.cfl_dt(U, 0.2))
        assert gm.sync_status() == 0
        assert _rel(Ug.cpu().numpy(), Uo).max() <= TOL


@pytest.mark.parametrize("system,flux,limiter,n,kind", [(0, 0, 0, 4, "wave"), (1, 1, 1, 5, "blast"),
                                                       (1, 1, 2, 3, "blast"), (0, 1, 1, 6, "kh")])
def test_fp64_path_is_bitwise_equal_to_oracle(pkg, system, flux, limiter, n, kind):
    """The FP64 path evaluates the same IEEE operations in the same order as the
    oracle (no contraction, identical tables and sums), so five CFL steps give
    identical bits, troubled flags and time steps."""
    import torch
    lo, hi = ((-0.5,) * 3, (0.5,) * 3) if kind == "kh" else ((0, 0, 0), (1, 1, 1))
    om, gm = _pair(pkg, system=system, K=(4, 3, 5), n=n, flux=flux, limiter=limiter, lo=lo, hi=hi)
    U = _init(om, kind)
    Ug = _gpu(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    tg = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    for _ in range(5):
        h = om.cfl_dt(U, 0.2)
        to = np.zeros(om.E, dtype=np.uint8)
        U = om.rk3_step(U, h, to)
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt, troubled=tg)
        assert dt.item() == h
        assert np.array_equal(tg.cpu().numpy(), to)
    assert gm.sync_status() == 0
    assert np.array_equal(Ug.cpu().numpy(), U)


def test_deterministic(pkg):
    om, gm = _pair(pkg, system=1, K=(4, 4, 4), n=5, flux=1, limiter=1)
    U = _init(om, "blast")
    a, b = _gpu(U), _gpu(U)
    for _ in range(3):
        gm.rk3_step(a, cfl=0.2)
        gm.rk3_step(b, cfl=0.2)
    assert bool((a == b).all())


def test_unphysical_state_reports_status(pkg):
    """A node with tau < 0 makes con2prim fail; the status word reports it and the
    kernels return normally (nothing traps)."""
    om, gm = _pair(pkg, system=1, K=(2, 2, 2), n=3, flux=1)
    U = _init(om, "blast")
    U[3, 4, 5] = -1.0
    R = gm.rhs(_gpu(U))
    assert gm.sync_status() == pkg.abi.DG_ERR_C2P
    assert gm.sync_status() == 0  # cleared


def _full_size_ten_steps(pkg, kw, kind):
    """Ten CFL steps at full size on both sides, in the launch configuration the
    bench times: the FP64 path bitwise equal to the oracle (dt of every step, the
    last step's troubled flags, the state); the mixed path, stepped on the
    oracle's dt sequence, within the mixed bar of 1e-6 relative L2 per conserved
    variable (LGL quadrature, each norm floored at 1 % of the largest; Sec. 3.4,
    SSP-RK3 with the limiter after every stage)."""
    import torch
    om, gm = _pair(pkg, **kw)
    U0 = _init(om, kind, seed=1)
    Ug = _gpu(U0)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    tg = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    U, hs = U0, []
    for _ in range(10):
        h = om.cfl_dt(U, 0.2)
        to = np.zeros(om.E, dtype=np.uint8)
        U = om.rk3_step(U, h, to)
        hs.append(h)
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt, troubled=tg)
        assert dt.item() == h
    assert gm.sync_status() == 0
    assert np.array_equal(tg.cpu().numpy(), to)
    assert np.array_equal(Ug.cpu().numpy(), U)
    del gm, Ug
    mm = pkg.Mesh(precision=1, **kw)
    Um = _gpu(U0)
    tm = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    for h in hs:
        mm.rk3_step(Um, dt=h, troubled=tm)
    assert mm.sync_status() == 0
    got = Um.cpu().numpy()
    _, d = om.norms(got, U)
    _, ref = om.norms(U, np.zeros_like(U))
    rel = d / np.maximum(ref, 1e-2 * ref.max())
    assert np.all(rel <= 1e-6), rel
    # the limiter decides the same way on all but a few elements (its 1e-8 face
    # test sits at the FP32 level of the mixed right-hand side)
    flips = np.count_nonzero(tm.cpu().numpy() != to)
    assert flips <= 1e-3 * om.E, flips


def test_full_size_blast_ten_steps(pkg):
    """The SR blast at full size (16^3 elements, n = 5, HLL, MinModN)."""
    _full_size_ten_steps(pkg, dict(system=1, K=(16, 16, 16), n=5, flux=1, limiter=1, gamma=4.0 / 3.0), "blast")


def test_full_size_con2prim_2p24(pkg):
    """The standalone con2prim workload at full size (2^24 seeded states): the
    GPU's primitives and iteration counts are bitwise the oracle's on every node."""
    import torch
    g = 4.0 / 3.0
    N = 1 << 24
    prim = di.c2p_samples(3, N, gamma=g)
    cons = oracle.prim2con(1, g, prim)
    del prim
    po, ito, sto = oracle.con2prim(g, cons)
    pg = torch.empty((5, N), dtype=torch.float64, device="cuda")
    it = torch.empty(N, dtype=torch.int32, device="cuda")
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    pkg.abi.dg_con2prim(N, g, _gpu(cons), pg, None, it, st)
    assert np.array_equal(st.cpu().numpy(), sto) and np.all(sto == 0)
    assert np.array_equal(pg.cpu().numpy(), po)
    assert np.array_equal(it.cpu().numpy(), ito)


def test_full_size_kh_ten_steps(pkg):
    """The Kelvin-Helmholtz workload at full size (64^3 elements, n = 6, HLL,
    MinModN; 56.6 M nodes)."""
    _full_size_ten_steps(pkg, dict(system=0, K=(64, 64, 64), n=6, flux=1, limiter=1, gamma=5.0 / 3.0,
                                   lo=(-0.5,) * 3, hi=(0.5,) * 3), "kh")


@pytest.mark.parametrize("n,limiter", [(2, 2), (4, 1), (6, 0)])
def test_roe_fp64_bitwise(pkg, n, limiter):
    """Roe flux (Sec. 3.2.3) on the FP64 path: RHS and three CFL steps of the
    shear layer bitwise equal to the oracle."""
    import torch
    kw = dict(system=0, K=(3, 2, 2), n=n, flux=2, limiter=limiter, gamma=5.0 / 3.0, lo=(-0.5,) * 3, hi=(0.5,) * 3)
    om, gm = _pair(pkg, **kw)
    U = _init(om, "kh", seed=2)
    assert np.array_equal(gm.rhs(_gpu(U)).cpu().numpy(), om.rhs(U))
    Ug = _gpu(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt)
        assert dt.item() == h
    assert gm.sync_status() == 0
    assert np.array_equal(Ug.cpu().numpy(), U)


def test_roe_rejected_for_sr(pkg):
    with pytest.raises(pkg.abi.DGError):
        pkg.Mesh(system=1, K=(2, 2, 2), n=3, flux=2, gamma=4.0 / 3.0)


@pytest.mark.parametrize("system,flux,limiter,n,kind", [(1, 1, 1, 4, "blast"), (0, 1, 0, 5, "kh"), (0, 2, 2, 3, "kh")])
def test_ab3_fp64_bitwise(pkg, system, flux, limiter, n, kind):
    """Adams-Bashforth (Sec. 3.4) on the FP64 path: six fixed-dt steps (two SSP-RK3
    start-up steps, then AB3 with the limiter and the fix) give the oracle's bits."""
    import torch
    kw = dict(system=system, K=(3, 3, 2), n=n, flux=flux, limiter=limiter)
    if kind == "kh":
        kw.update(gamma=5.0 / 3.0, lo=(-0.5,) * 3, hi=(0.5,) * 3)
    om, gm = _pair(pkg, **kw)
    U = _init(om, kind, seed=2)
    dt = 0.5 * om.cfl_dt(U, 0.2)
    Uo = om.ab3_run(U, 6, dt)
    Ug = _gpu(U)
    for _ in range(6):
        gm.ab3_step(Ug, dt)
    assert gm.sync_status() == 0
    assert np.array_equal(Ug.cpu().numpy(), Uo)
    with pytest.raises(pkg.abi.DGError):
        gm.ab3_step(Ug, 0.5 * dt)
    gm.ab3_reset()
    gm.ab3_step(Ug, 0.5 * dt)
