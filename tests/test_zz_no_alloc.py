"""dg_rhs_static: the FP64 right-hand side for callers that cannot allocate
device memory (their memory belongs to another allocator, or they cannot afford
cudaMalloc's device synchronisation).  It must give exactly what dg_rhs gives on
a mesh built from the same descriptor, call after call, although its scratch
lives in one static device array shared by every call.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import dg_inputs as di
import oracle

pytestmark = pytest.mark.gpu


def test_rhs_static_equals_rhs_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as pkg
    from paper_1609_00098_gb300 import build as b
    b.build()
    cases = [dict(system=1, K=(5, 4, 3), n=5, flux=1, gamma=4.0 / 3.0),
             dict(system=0, K=(3, 3, 3), n=4, flux=0, gamma=1.4),
             dict(system=0, K=(4, 2, 3), n=6, flux=2, gamma=1.4)]  # the Roe flux, as dg_rhs accepts it
    for kw in cases:
        desc = pkg.make_desc(**kw)
        mesh = pkg.Mesh(**kw)
        om = oracle.Mesh(oracle.MeshSpec(**kw))
        xyz = om.coords()
        for seed in (1, 2):  # two calls in a row: the static scratch keeps the previous call's data
            prim = di.blast_sr(xyz, seed=seed) if kw["system"] == 1 else di.smooth_wave_ne(xyz, k=(seed, 1, 2))
            U = torch.from_numpy(om.from_prim(prim)).cuda()
            ref = mesh.rhs(U)
            out = torch.full_like(U, float("nan"))
            pkg.abi.dg_rhs_static(desc, U, out)
            torch.cuda.synchronize()
            # same kernels, same operation order: identical bits (the FP64 tolerance is exactness)
            assert torch.equal(out, ref)
        mesh.close()


def test_rhs_static_rejects_meshes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as pkg
    desc = pkg.make_desc(system=0, K=(20, 16, 16), n=3)  # 5,120 elements * 27 nodes = 138,240 > 131,072
    U = torch.zeros(20 * 16 * 16 * 27 * 5, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DGError) as ei:
        pkg.abi.dg_rhs_static(desc, U, U.clone())
    assert ei.value.status == pkg.abi.DG_ERR_ARG


def test_rhs_static_allocates_nothing_after_its_first_call():
    """Free device memory stays the same over repeated calls (the first call on a
    device may load the library's module and look up the array's address)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as pkg
    kw = dict(system=0, K=(4, 4, 4), n=4, flux=1, gamma=1.4)
    desc = pkg.make_desc(**kw)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    U = torch.from_numpy(om.from_prim(di.smooth_wave_ne(om.coords(), k=(1, 2, 1)))).cuda()
    out = torch.empty_like(U)
    pkg.abi.dg_rhs_static(desc, U, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        pkg.abi.dg_rhs_static(desc, U, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rhs_static_unphysical_node_gives_non_finite_rhs():
    """A node without a physical primitive state (SR, tau < 0) has no status word
    to report it through this entry point: it shows as non-finite values of dU/dt
    in its element, as the header documents; other elements away from it stay
    finite."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as pkg
    kw = dict(system=1, K=(4, 3, 3), n=3, flux=1, gamma=4.0 / 3.0)
    desc = pkg.make_desc(**kw)
    om = oracle.Mesh(oracle.MeshSpec(**kw))
    U0 = om.from_prim(di.blast_sr(om.coords(), seed=1))
    bad = 13  # element (1, 0, 1)
    U0[bad, 4, 5] = -1.0
    U = torch.from_numpy(U0).cuda()
    out = torch.zeros_like(U)
    pkg.abi.dg_rhs_static(desc, U, out)
    torch.cuda.synchronize()
    R = out.cpu().numpy()
    assert not np.all(np.isfinite(R[bad]))
    far = 4 * 3 * 3 - 1  # element (3, 2, 2): no face shared with element (1, 0, 1)
    assert np.all(np.isfinite(R[far]))
