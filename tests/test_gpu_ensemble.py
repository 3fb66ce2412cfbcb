"""Ragged ensemble: meshes of different n, K and systems advanced together by
per-group batched launches (and a replayed CUDA graph) give the same bits as
stepping each mesh on its own, before and after the launch-shape autotuner."""
import numpy as np
import pytest

import dg_inputs as di
from oracle import mlp

pytestmark = pytest.mark.gpu

SPECS = [  # (system, K, n, flux, limiter, learned)
    (0, (3, 3, 3), 3, 0, 0, False),
    (0, (2, 3, 2), 4, 0, 0, False),
    (0, (2, 2, 2), 3, 0, 0, False),   # same group as the first
    (1, (3, 3, 3), 5, 1, 1, False),
    (1, (4, 2, 2), 4, 1, 1, False),
    (1, (2, 3, 2), 5, 1, 1, True),
    (0, (2, 2, 2), 6, 1, 1, False),
]


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_00098_gb300 as p
    from paper_1609_00098_gb300 import build as b
    b.build()
    return p


@pytest.fixture(scope="module")
def net(pkg):
    p = mlp.init_params(di.uniform(5, 9, np.arange(mlp.N_PARAMS))).astype(np.float32)
    h = pkg.abi.dg_c2p_net_create(p, mlp.DEFAULT_SCALES)
    yield h
    pkg.abi.dg_c2p_net_destroy(h)


def _make(pkg, net):
    import torch
    meshes, states = [], []
    for system, K, n, flux, lim, learned in SPECS:
        g = 4.0 / 3.0 if system else 1.4
        m = pkg.Mesh(system=system, K=K, n=n, flux=flux, limiter=lim, gamma=g, precision=1)
        if learned:
            m.set_c2p_net(net)
        xyz = m.coords().cpu().numpy()
        prim = di.blast_sr(xyz, seed=3) if system else di.smooth_wave_ne(xyz, k=di.wave_numbers(3))
        states.append(m.from_prim(torch.from_numpy(prim).cuda()))
        meshes.append(m)
    return meshes, states


def _run_ensemble(pkg, meshes, states, steps, tune):
    import torch
    ens = pkg.abi.dg_ensemble_create([m.h for m in meshes], states)
    try:
        if tune:
            pkg.abi.dg_ensemble_tune(ens)
        groups = pkg.abi.dg_ensemble_groups(ens)
        for k in range(steps):
            # direct launches, graph with the groups on one chain, graph with the
            # groups on parallel branches: the same bits
            pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=(0, 1, 2, 1)[k % 4])
        dt = torch.empty(len(meshes), dtype=torch.float64, device="cuda")
        pkg.abi.dg_ensemble_dt(ens, dt)
        torch.cuda.synchronize()
        return groups, dt.cpu().numpy()
    finally:
        pkg.abi.dg_ensemble_destroy(ens)


@pytest.mark.parametrize("tune", [False, True])
def test_ensemble_matches_meshes_one_by_one(pkg, net, tune):
    import torch
    em, es = _make(pkg, net)
    rm, rs = _make(pkg, net)
    groups, dt_e = _run_ensemble(pkg, em, es, 4, tune)
    assert len(groups) == 6 and sum(g["meshes"] for g in groups) == len(SPECS)
    # the reference meshes take the contraction each group ended up with
    for g in groups:
        for i in g["members"]:
            rm[i].set_option(pkg.abi.OPT_TENSOR_CORE_CONTRACTION, g["tc"])
    dt_r = np.zeros(len(SPECS))
    dtv = torch.zeros(1, dtype=torch.float64, device="cuda")
    for i, m in enumerate(rm):
        for _ in range(4):
            m.rk3_step(rs[i], cfl=0.2, dt_used=dtv)
        dt_r[i] = float(dtv.item())
    for i in range(len(SPECS)):
        assert em[i].sync_status() == 0 and rm[i].sync_status() == 0
        assert torch.equal(es[i], rs[i]), (i, SPECS[i], float((es[i] - rs[i]).abs().max()))
    assert np.array_equal(dt_e, dt_r), (dt_e, dt_r)
    if tune:
        for g in groups:
            assert 1 <= g["epb"] and g["tc"] in (0, 1)


def test_ensemble_rejects_bad_members(pkg):
    import torch
    m64 = pkg.Mesh(system=0, K=(2, 2, 2), n=3, precision=0)
    mm = pkg.Mesh(system=0, K=(2, 2, 2), n=3, precision=1)
    U = mm.state()
    with pytest.raises(pkg.abi.DGError):
        pkg.abi.dg_ensemble_create([m64.h], [m64.state()])
    with pytest.raises(pkg.abi.DGError):
        pkg.abi.dg_ensemble_create([mm.h, mm.h], [U, torch.zeros_like(U)])


# (system, K, n, flux, limiter, learned): both systems, extreme n, a K = 1 axis.  The
# self-periodic axis is on a member without the limiter: there the neighbours' means
# are the element's own, MinModN's face test reduces to |U0 - face mean| <= 1e-8,
# and on the smooth wave that gap is zero in exact arithmetic but FP32 rounding of
# the mixed right-hand side at n = 7, 8 (~1e-7) exceeds it.
ORACLE_SPECS = [
    (0, (3, 2, 1), 2, 0, 0, False),
    (0, (2, 2, 2), 8, 1, 1, False),
    (0, (3, 3, 2), 5, 1, 1, False),
    (1, (3, 2, 2), 3, 1, 1, False),
    (1, (2, 3, 2), 5, 1, 1, True),
    (1, (2, 2, 2), 4, 0, 1, False),
]


def test_ensemble_matches_oracle(pkg, net):
    """Every member of a ragged ensemble, advanced by the batched launches (graph
    replayed after the first step), against the FP64 oracle stepped on the same
    dt sequence (each step's dt read back with dg_ensemble_dt): within the mixed
    bar, 1e-6 relative L2 per conserved variable (LGL quadrature, each norm
    floored at 1 % of the largest) after five SSP-RK3 steps (Sec. 3.4)."""
    import torch
    import oracle
    meshes, states, oms, Uo = [], [], [], []
    for system, K, n, flux, lim, learned in ORACLE_SPECS:
        g = 4.0 / 3.0 if system else 1.4
        om = oracle.Mesh(oracle.MeshSpec(system=system, K=K, n=n, flux=flux, limiter=lim, gamma=g))
        xyz = om.coords()
        U0 = om.from_prim(di.blast_sr(xyz, seed=2) if system else di.smooth_wave_ne(xyz, k=(1, 2, 1)))
        m = pkg.Mesh(system=system, K=K, n=n, flux=flux, limiter=lim, gamma=g, precision=1)
        if learned:
            m.set_c2p_net(net)
        meshes.append(m)
        states.append(torch.from_numpy(U0).cuda())
        oms.append(om)
        Uo.append(U0)
    ens = pkg.abi.dg_ensemble_create([m.h for m in meshes], states)
    try:
        dt = torch.empty(len(meshes), dtype=torch.float64, device="cuda")
        for k in range(5):
            pkg.abi.dg_ensemble_step(ens, 0.2, use_graph=True)
            pkg.abi.dg_ensemble_dt(ens, dt)
            h = dt.cpu().numpy()
            for i, om in enumerate(oms):
                Uo[i] = om.rk3_step(Uo[i], float(h[i]))
    finally:
        pkg.abi.dg_ensemble_destroy(ens)
    for i, om in enumerate(oms):
        assert meshes[i].sync_status() == 0
        got = states[i].cpu().numpy()
        _, d = om.norms(got, Uo[i])
        _, ref = om.norms(Uo[i], np.zeros_like(Uo[i]))
        rel = d / np.maximum(ref, 1e-2 * ref.max())
        assert np.all(rel <= 1e-6), (i, ORACLE_SPECS[i], rel)


def test_ensemble_step_rejects_bad_arguments(pkg, net):
    em, es = _make(pkg, net)
    ens = pkg.abi.dg_ensemble_create([m.h for m in em], es)
    try:
        for cfl, mode in ((0.0, 1), (0.2, 3), (0.2, -1)):
            with pytest.raises(pkg.abi.DGError):
                pkg.abi.dg_ensemble_step(ens, cfl, use_graph=mode)
    finally:
        pkg.abi.dg_ensemble_destroy(ens)
        for m in em:
            m.close()
