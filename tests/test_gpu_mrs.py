"""Moment limiter of Moe, Rossmanith and Seal (Sec. 3.3.3) on the GPU: the FP64
path gives the oracle's bits (limiter alone, SSP-RK3 and Adams-Bashforth steps,
the troubled-cell mask included); the mixed path stays within the 1e-6 bar."""
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


def _case(kind, n, alpha, flux=2, precision=0, K=None):
    """(oracle mesh kwargs, GPU mesh kwargs, initial state builder)."""
    if kind == "sod":
        kw = dict(system=0, K=K or (8, 2, 2), n=n, flux=flux, limiter=3, gamma=1.4, lo=(-1, 0, 0), hi=(1, 1, 1),
                  mrs_alpha=alpha)
        init = lambda om: om.from_prim(di.riemann_1d(om.coords(), "sod"))  # noqa: E731
    else:
        kw = dict(system=0, K=K or (4, 3, 2), n=n, flux=flux, limiter=3, gamma=5.0 / 3.0, lo=(-0.5,) * 3,
                  hi=(0.5,) * 3, mrs_alpha=alpha)
        init = lambda om: om.from_prim(di.kh_ne(om.coords(), seed=2))  # noqa: E731
    return kw, dict(kw, precision=precision), init


@pytest.mark.parametrize("n,alpha,kind", [(2, 0.0, "sod"), (3, 0.5, "kh"), (5, 0.0, "kh"), (8, 2.0, "sod")])
@pytest.mark.parametrize("precision", [0, 1])
def test_mrs_limit_alone_bitwise(pkg, n, alpha, kind, precision):
    """dg_limit with the moment limiter: the limited state and the troubled mask
    equal the oracle's bit for bit (both precisions run the FP64 limiter here)."""
    import torch
    kw, gkw, init = _case(kind, n, alpha, precision=precision)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    gm = pkg.Mesh(**gkw)
    U = init(om)
    # one unlimited-looking step of the oracle gives a state with new extrema
    U = U + 0.05 * om.rhs(U) * om.cfl_dt(U, 0.2)
    Uo, to = om.limit(U)
    Ug = _gpu(U)
    tg = torch.zeros(gm.E, dtype=torch.uint8, device="cuda")
    gm.limit(Ug, troubled=tg)
    assert gm.sync_status() == 0
    assert int(to.astype(bool).sum()) > 0
    assert np.array_equal(tg.cpu().numpy(), to)
    assert np.array_equal(Ug.cpu().numpy(), Uo)


@pytest.mark.parametrize("flux,n,alpha,kind", [(2, 3, 0.5, "sod"), (0, 4, 0.0, "kh"), (1, 2, 1.0, "kh")])
def test_mrs_rk3_fp64_bitwise(pkg, flux, n, alpha, kind):
    """Five CFL SSP-RK3 steps with the moment limiter after every stage: state,
    dt and the last stage's troubled mask equal the oracle's."""
    import torch
    kw, gkw, init = _case(kind, n, alpha, flux=flux)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    gm = pkg.Mesh(**gkw)
    U = init(om)
    Ug = _gpu(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    tg = torch.zeros(gm.E, dtype=torch.uint8, device="cuda")
    to = np.zeros(om.E, dtype=np.uint8)
    for _ in range(5):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h, troubled=to)
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt, troubled=tg)
        assert dt.item() == h
    assert gm.sync_status() == 0
    assert np.array_equal(tg.cpu().numpy(), to)
    assert np.array_equal(Ug.cpu().numpy(), U)


def test_mrs_ab3_fp64_bitwise(pkg):
    kw, gkw, init = _case("sod", 3, 0.5)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    gm = pkg.Mesh(**gkw)
    U = init(om)
    dt = 0.5 * om.cfl_dt(U, 0.2)
    Uo = om.ab3_run(U, 6, dt)
    Ug = _gpu(U)
    for _ in range(6):
        gm.ab3_step(Ug, dt)
    assert gm.sync_status() == 0
    assert np.array_equal(Ug.cpu().numpy(), Uo)


def _rel_l2(om, a, b):
    _, d = om.norms(a, b)
    _, ref = om.norms(b, np.zeros_like(b))
    return d / np.maximum(ref, 1e-2 * ref.max())


@pytest.mark.parametrize("flux,n,kind", [(2, 3, "sod"), (1, 5, "kh")])
def test_mrs_mixed_close_to_oracle(pkg, flux, n, kind):
    """Mixed precision (FP32 right-hand side, FP64 accumulation and FP64 moment
    limiter): ten steps on the oracle's dt sequence within 1e-6 relative L2."""
    kw, gkw, init = _case(kind, n, 0.5, flux=flux, precision=1)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    gm = pkg.Mesh(**gkw)
    U = init(om)
    Ug = _gpu(U)
    for _ in range(10):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


def test_mrs_rejections(pkg):
    with pytest.raises(pkg.abi.DGError):
        pkg.Mesh(system=1, K=(2, 2, 2), n=3, flux=1, limiter=3, gamma=4.0 / 3.0)
    with pytest.raises(pkg.abi.DGError):
        pkg.Mesh(system=0, K=(2, 2, 2), n=3, limiter=3, mrs_alpha=-1.0)
    m = pkg.Mesh(system=0, K=(2, 2, 2), n=3, limiter=3, precision=1)
    with pytest.raises(pkg.abi.DGError):
        pkg.abi.dg_ensemble_create([m.h], [m.state()])
