"""Mixed-precision path (FP32 arithmetic, FP64 state and accumulation) against
the FP64 oracle.  Bars: on the smooth problem with an exact solution, the mixed
L2 error stays within 1.05x of the oracle's; without an exact solution (blast,
Kelvin-Helmholtz) the relative L2 distance to the oracle stays within 1e-6 per
conserved variable.  A variable's norm is floored at 1 % of the largest
variable's norm: momenta that start at zero (blast at rest, S_z of the shear
layer) have no scale of their own."""
import numpy as np
import pytest

import dg_inputs as di
import oracle

pytestmark = pytest.mark.gpu


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


def _pair(pkg, system, K, n, flux, limiter, lo=(0, 0, 0), hi=(1, 1, 1), gamma=None):
    gamma = gamma or (1.4 if system == 0 else 4.0 / 3.0)
    om = oracle.Mesh(oracle.MeshSpec(system=system, K=K, n=n, flux=flux, limiter=limiter, gamma=gamma, lo=lo, hi=hi))
    gm = pkg.Mesh(system=system, K=K, n=n, flux=flux, limiter=limiter, gamma=gamma, lo=lo, hi=hi, precision=1)
    return om, gm


def _rel_l2(om, a, b):
    """Per-variable relative L2 distance with LGL quadrature (norm floored at 1 %
    of the largest variable's norm)."""
    _, d = om.norms(a, b)
    _, ref = om.norms(b, np.zeros_like(b))
    scale = np.maximum(ref, 1e-2 * ref.max())
    return d / scale


def _scale(R):
    m = np.abs(R).max(axis=(0, 2))
    return np.maximum(m, 1e-2 * m.max())


@pytest.mark.parametrize("system,flux,n,kind", [(0, 0, 4, "wave"), (1, 1, 5, "blast"), (0, 1, 6, "kh"),
                                                (1, 0, 3, "re_smooth")])
def test_mixed_rhs_close_to_oracle(pkg, system, flux, n, kind):
    lo, hi = ((-0.5,) * 3, (0.5,) * 3) if kind == "kh" else ((0, 0, 0), (1, 1, 1))
    om, gm = _pair(pkg, system, (4, 3, 3), n, flux, 0, lo, hi)
    xyz = om.coords()
    prim = {"wave": lambda: di.smooth_wave_ne(xyz, k=(1, 2, 1)), "blast": lambda: di.blast_sr(xyz, seed=1),
            "kh": lambda: di.kh_ne(xyz, seed=1), "re_smooth": lambda: di.smooth_flow_re(xyz, gamma=4 / 3)}[kind]()
    U = om.from_prim(prim)
    Ro = om.rhs(U)
    Rg = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    # FP32 arithmetic: relative max-norm error of the RHS at the level of a few FP32 ulps
    # times the ratio of flux to RHS magnitudes
    err = np.abs(Rg - Ro).max(axis=(0, 2)) / _scale(Ro)
    assert err.max() < 5e-4, err


def test_mixed_smooth_wave_error_within_5_percent_of_fp64(pkg):
    """Configuration 1 (Newtonian smooth wave, K=4, n=4, Rusanov, 10 CFL steps):
    the mixed path's L2 error against the exact solution is within 1.05x of the
    FP64 oracle's."""
    import torch
    om, gm = _pair(pkg, 0, (4, 4, 4), 4, 0, 0)
    k = di.wave_numbers(1)
    U0 = om.from_prim(di.smooth_wave_ne(om.coords(), k=k))
    Uo, t = U0.copy(), 0.0
    dts = []
    for _ in range(10):
        h = om.cfl_dt(Uo, 0.2)
        dts.append(h)
        Uo = om.rk3_step(Uo, h)
        t += h
    Ug = _gpu(U0)
    for h in dts:
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    Uex = om.from_prim(di.smooth_wave_ne(om.coords(), t, k=k))
    eo = om.norms(Uo, Uex)[1]
    eg = om.norms(Ug.cpu().numpy(), Uex)[1]
    assert np.all(eg <= 1.05 * eo + 1e-12), (eg, eo)
    # and the CFL step computed on the device in FP32 agrees with the FP64 one
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    Ug2 = _gpu(U0)
    gm.rk3_step(Ug2, cfl=0.2, dt_used=dt)
    assert abs(dt.item() - dts[0]) <= 1e-6 * dts[0]


@pytest.mark.parametrize("limiter", [1, 2])
def test_mixed_blast_close_to_oracle(pkg, limiter):
    """SR blast with HLL and a limiter after every stage: after 10 steps with the
    oracle's time steps, relative L2 distance to the FP64 oracle <= 1e-6."""
    om, gm = _pair(pkg, 1, (6, 5, 5), 5, 1, limiter)
    U = om.from_prim(di.blast_sr(om.coords(), seed=1))
    Ug = _gpu(U)
    for _ in range(10):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


@pytest.mark.parametrize("limiter", [0, 1])
def test_mixed_cold_fast_flow_fix_everywhere(pkg, limiter):
    """A cold SR flow at |v| ~ 0.9 (p = 1e-10 rho, 2 % density noise): S^2 sits
    within 1e-10 of tau (tau + 2D) at every node, so the conserved fix of Sec. 2.1.4
    acts at most nodes after the first stage (77 %, oracle count), and with the
    limiter every node of every element goes through its FP64 check.  After three
    steps at the oracle's time steps, relative L2 distance to the oracle <= 1e-6."""
    om, gm = _pair(pkg, 1, (4, 3, 3), 5, 1, limiter)
    xyz = om.coords()
    u = di.uniform(7, 0, np.arange(xyz[0].size)).reshape(xyz[0].shape)
    rho = 1.0 + 0.02 * (u - 0.5)
    prim = np.stack([rho, np.full_like(rho, 0.9), 0.1 * np.sin(2 * np.pi * xyz[0]), np.zeros_like(rho),
                     1e-10 * rho])
    U = om.from_prim(prim)
    Ug = _gpu(U)
    for _ in range(3):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


def test_mixed_kh_close_to_oracle(pkg):
    om, gm = _pair(pkg, 0, (4, 4, 4), 6, 1, 1, lo=(-0.5,) * 3, hi=(0.5,) * 3, gamma=5 / 3)
    U = om.from_prim(di.kh_ne(om.coords(), seed=1))
    Ug = _gpu(U)
    for _ in range(10):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


@pytest.mark.parametrize("n,flux,limiter,K", [(3, 0, 2, (5, 4, 3)), (7, 1, 2, (3, 3, 2)), (4, 2, 1, (9, 2, 3)),
                                             (8, 1, 1, (2, 3, 2))])
def test_mixed_ne_difference_form(pkg, n, flux, limiter, K):
    """The Newtonian difference-form step (SSP-RK3 of Sec. 3.4 written in stage
    differences, the limiter's summaries by linearity, Sec. 3.3.1-3.3.2) with
    MinMod and MinModN, LLF, HLL and Roe, odd and even n, element counts that are
    not multiples of the elements per CTA: five shear-layer steps within the
    1e-6 bar of the oracle, and the last stage's troubled flags equal."""
    import torch
    kw = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, gamma=5 / 3)
    om, gm = _pair(pkg, 0, K, n, flux, limiter, **kw)
    U = om.from_prim(di.kh_ne(om.coords(), seed=4))
    Ug = _gpu(U)
    tg = torch.zeros(om.E, dtype=torch.uint8, device="cuda")
    for _ in range(5):
        h = om.cfl_dt(U, 0.2)
        to = np.zeros(om.E, dtype=np.uint8)
        U = om.rk3_step(U, h, to)
        gm.rk3_step(Ug, dt=h, troubled=tg)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d
    if limiter == 2:
        assert np.all(tg.cpu().numpy() == 0x1f) and np.all(to == 0x1f)  # MinMod limits every variable


def test_mixed_ne_state_not_16_byte_aligned_is_refused(pkg):
    """The mixed Newtonian kernels move the FP64 state in 16-byte pieces (vector
    loads and stores, bulk copies into shared memory), so a caller's U that starts
    8 bytes past a 16-byte boundary is refused with DG_ERR_ARG before anything is
    launched; the same state at an aligned address steps normally."""
    import torch
    kw = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, gamma=5 / 3)
    om, gm = _pair(pkg, 0, (4, 3, 2), 6, 1, 1, **kw)
    U0 = om.from_prim(di.kh_ne(om.coords(), seed=5))
    buf = torch.empty(U0.size + 1, dtype=torch.float64, device="cuda")
    Ub = buf[1:].view(U0.shape)
    Ub.copy_(_gpu(U0))
    assert Ub.data_ptr() % 16 == 8
    h = om.cfl_dt(U0, 0.2)
    for call in (lambda: gm.rk3_step(Ub, dt=h), lambda: gm.rhs(Ub)):
        with pytest.raises(pkg.abi.DGError) as ei:
            call()
        assert ei.value.status == pkg.abi.DG_ERR_ARG
    with pytest.raises(pkg.abi.DGError):
        pkg.abi.dg_ensemble_create([gm.h], [Ub])
    Ua = _gpu(U0)
    gm.rk3_step(Ua, dt=h)
    assert gm.sync_status() == 0


def test_mixed_conservation(pkg):
    """FP64 state: totals drift only by the FP32 rounding of the fluxes and of the
    stage increments (relative to the largest total)."""
    om, gm = _pair(pkg, 1, (4, 4, 4), 4, 1, 1)
    U = om.from_prim(di.blast_sr(om.coords(), seed=2))
    t0 = om.totals(U)
    Ug = _gpu(U)
    for _ in range(5):
        gm.rk3_step(Ug, cfl=0.2)
    t1 = om.totals(Ug.cpu().numpy())
    assert gm.sync_status() == 0
    drift = np.abs(t1 - t0) / np.abs(t0).max()
    assert np.all(drift < 1e-7), drift


def test_mixed_ill_conditioned_nodes(pkg):
    """Fast cold flow (W ~ 8, eps ~ 1e-6): FP32 con2prim alone would lose the
    pressure; the FP64 polish keeps the RHS at FP32 accuracy."""
    om, gm = _pair(pkg, 1, (3, 3, 3), 4, 1, 0)
    x, y, z = om.coords()
    v = 0.99 + 0.002 * np.sin(2 * np.pi * x)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * y)
    p = (1.0 / 3.0) * rho * 1e-6
    prim = np.stack([rho, v, 0 * v, 0 * v, p])
    U = om.from_prim(prim)
    Ro = om.rhs(U)
    Rg = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    err = np.abs(Rg - Ro).max(axis=(0, 2)) / _scale(Ro)
    assert err.max() < 1e-3, err


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_tensor_core_and_fma_contractions(pkg, n):
    """The volume contraction on the tensor cores (split-BF16x3, FP32 accumulate)
    and on the CUDA cores (FP32 FMA) both give the oracle's RHS to FP32 rounding,
    and agree with each other to the same level."""
    om, gm = _pair(pkg, 1, (3, 2, 2), n, 1, 1)
    U = om.from_prim(di.blast_sr(om.coords(), seed=4))
    Ro = om.rhs(U)
    out = {}
    for tc in (1, 0):
        gm.set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, tc)
        out[tc] = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    sc = _scale(Ro)
    for tc in (1, 0):
        err = np.abs(out[tc] - Ro).max(axis=(0, 2)) / sc
        assert err.max() < 1e-4, (tc, err)
    diff = np.abs(out[1] - out[0]).max(axis=(0, 2)) / sc
    assert diff.max() < 1e-4, diff


def test_mesh_options_validate(pkg):
    gm = pkg.Mesh(system=1, K=(2, 2, 2), n=3, flux=1, limiter=0, precision=1, gamma=4.0 / 3.0)
    for opt, bad in ((pkg.abi.OPT_TENSOR_CORE_CONTRACTION, 2), (pkg.abi.OPT_C2P_KAPPA_SWITCH, 0.5), (99, 1)):
        with pytest.raises(pkg.abi.DGError):
            gm.set_option(opt, bad)
    gm.set_option(pkg.abi.OPT_C2P_KAPPA_SWITCH, 1e3)
    gm.set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, 0)
    for bad in (0, 3, 16):
        with pytest.raises(pkg.abi.DGError):
            gm.set_option(pkg.abi.OPT_ELEMENTS_PER_CTA, bad)
    gm.set_option(pkg.abi.OPT_ELEMENTS_PER_CTA, 8)


@pytest.mark.parametrize("n,epb", [(3, 4), (4, 2), (5, 2)])
def test_elements_per_cta_do_not_change_results(pkg, n, epb):
    """Several elements per CTA (the learned guess batched over all of them)
    give the same bits as one element per CTA."""
    from oracle import mlp
    net = pkg.abi.dg_c2p_net_create(mlp.init_params(di.uniform(5, 9, np.arange(mlp.N_PARAMS))).astype(np.float32),
                                    mlp.DEFAULT_SCALES)
    try:
        out = []
        for e in (1, epb):
            om, gm = _pair(pkg, 1, (3, 3, 2), n, 1, 1)
            gm.set_c2p_net(net)
            gm.set_option(pkg.abi.OPT_ELEMENTS_PER_CTA, e)
            U = _gpu(om.from_prim(di.blast_sr(om.coords(), seed=2)))
            for _ in range(3):
                gm.rk3_step(U, cfl=0.2)
            assert gm.sync_status() == 0
            out.append(U.cpu().numpy())
        assert np.array_equal(out[0], out[1])
    finally:
        pkg.abi.dg_c2p_net_destroy(net)


@pytest.mark.parametrize("K,n,system,epb", [((1, 1, 1), 2, 0, 1), ((1, 3, 1), 8, 1, 1), ((7, 1, 2), 3, 1, 4),
                                            ((3, 1, 1), 5, 1, 2)])
def test_mixed_edge_case_shapes(pkg, K, n, system, epb):
    """Self-periodic K = 1 axes, ragged element counts (not a multiple of the
    stage kernel's elements per CTA nor of the limiter's warps per CTA),
    anisotropic boxes and both extreme n on the mixed path: two steps within the
    mixed bar (1e-6 relative L2) of the oracle."""
    om = oracle.Mesh(oracle.MeshSpec(system=system, K=K, n=n, flux=1, limiter=1, gamma=1.4 if system == 0 else 4 / 3,
                                     lo=(0, -2, 0), hi=(1, 1, 0.25)))
    gm = pkg.Mesh(system=system, K=K, n=n, flux=1, limiter=1, gamma=1.4 if system == 0 else 4 / 3,
                  lo=(0, -2, 0), hi=(1, 1, 0.25), precision=1)
    gm.set_option(pkg.abi.OPT_ELEMENTS_PER_CTA, epb)
    xyz = om.coords()
    U = om.from_prim(di.smooth_wave_ne(xyz, k=(1, 1, 1)) if system == 0 else di.blast_sr(xyz, seed=3))
    Ug = _gpu(U)
    for _ in range(2):
        h = 0.5 * om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


def test_mixed_roe(pkg):
    """Roe flux on the mixed path: RHS to FP32 rounding of the oracle's, and ten
    shear-layer steps within the 1e-6 bar."""
    om, gm = _pair(pkg, 0, (4, 4, 4), 5, 2, 1, lo=(-0.5,) * 3, hi=(0.5,) * 3, gamma=5 / 3)
    U = om.from_prim(di.kh_ne(om.coords(), seed=3))
    Ro = om.rhs(U)
    err = np.abs(gm.rhs(_gpu(U)).cpu().numpy() - Ro).max(axis=(0, 2)) / _scale(Ro)
    assert err.max() < 5e-4, err  # the FP32 level of test_mixed_rhs_close_to_oracle
    Ug = _gpu(U)
    for _ in range(10):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


def test_mixed_ab3_newtonian(pkg):
    """Adams-Bashforth on a mixed Newtonian mesh: the right-hand side of the
    difference-form kernel (dg_rhs) and its start-up steps (two SSP-RK3 steps in
    difference form), the combination in FP64; ten shear-layer steps within the
    1e-6 bar of the oracle's AB3 (Sec. 3.4)."""
    om, gm = _pair(pkg, 0, (4, 3, 3), 6, 1, 1, lo=(-0.5,) * 3, hi=(0.5,) * 3, gamma=5 / 3)
    U = om.from_prim(di.kh_ne(om.coords(), seed=2))
    dt = 0.5 * om.cfl_dt(U, 0.2)
    Uo = om.ab3_run(U, 10, dt)
    Ug = _gpu(U)
    for _ in range(10):
        gm.ab3_step(Ug, dt)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), Uo)
    assert np.all(d <= 1e-6), d


def test_mixed_ab3(pkg):
    """Adams-Bashforth on a mixed mesh (mixed right-hand side, FP64 combination):
    ten blast steps within the 1e-6 bar of the oracle's AB3."""
    om, gm = _pair(pkg, 1, (4, 3, 3), 5, 1, 1)
    U = om.from_prim(di.blast_sr(om.coords(), seed=1))
    dt = 0.5 * om.cfl_dt(U, 0.2)
    Uo = om.ab3_run(U, 10, dt)
    Ug = _gpu(U)
    for _ in range(10):
        gm.ab3_step(Ug, dt)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), Uo)
    assert np.all(d <= 1e-6), d
