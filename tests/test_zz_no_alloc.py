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
             dict(system=0, K=(3, 3, 3), n=4, flux=0, gamma=1.4)]
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
