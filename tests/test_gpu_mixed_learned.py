"""Mixed-precision path with the learned con2prim starting guess computed inside
the stage kernel (dg_mesh_set_c2p_net).  Newton still decides the result, so the same
bars as the warm-started mixed path hold: within 1e-6 relative L2 (per conserved
variable, norm floored at 1 % of the largest) of the FP64 oracle after 10 blast
steps, for a trained network and for an untrained one."""
import numpy as np
import pytest

import dg_inputs as di
import oracle
from oracle import mlp

pytestmark = pytest.mark.gpu

G = 4.0 / 3.0


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


def _params(seed):
    return mlp.init_params(di.uniform(seed, 9, np.arange(mlp.N_PARAMS))).astype(np.float32)


@pytest.fixture(scope="module")
def trained(pkg):
    """A network trained on 2^17 pairs the method generates (prim -> cons)."""
    prim = di.c2p_samples(41, 1 << 17, gamma=G)
    cons = oracle.prim2con(1, G, prim)
    net = pkg.abi.dg_c2p_net_create(_params(5), mlp.DEFAULT_SCALES)
    pkg.abi.dg_c2p_net_train(net, cons.shape[1], _gpu(cons), _gpu(prim[4]), 6, 2048, 2e-3)
    yield net
    pkg.abi.dg_c2p_net_destroy(net)


def _rel_l2(om, a, b):
    _, d = om.norms(a, b)
    _, ref = om.norms(b, np.zeros_like(b))
    return d / np.maximum(ref, 1e-2 * ref.max())


def _blast(pkg, limiter, net, steps=10):
    om = oracle.Mesh(oracle.MeshSpec(system=1, K=(6, 5, 5), n=5, flux=1, limiter=limiter, gamma=G))
    gm = pkg.Mesh(system=1, K=(6, 5, 5), n=5, flux=1, limiter=limiter, gamma=G, precision=1)
    gm.set_c2p_net(net)
    U = om.from_prim(di.blast_sr(om.coords(), seed=1))
    Ug = _gpu(U)
    for _ in range(steps):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    return _rel_l2(om, Ug.cpu().numpy(), U), Ug.cpu().numpy()


@pytest.mark.parametrize("limiter", [1, 2])
def test_learned_guess_blast_close_to_oracle(pkg, trained, limiter):
    d, _ = _blast(pkg, limiter, trained)
    assert np.all(d <= 1e-6), d


def test_untrained_guess_changes_only_iterations(pkg):
    """A network that has never been trained gives poor guesses; the Newton
    solves still converge to the same pressures within their stopping tolerance,
    so the result meets the same bar."""
    net = pkg.abi.dg_c2p_net_create(_params(6), mlp.DEFAULT_SCALES)
    try:
        d, _ = _blast(pkg, 1, net)
        assert np.all(d <= 1e-6), d
    finally:
        pkg.abi.dg_c2p_net_destroy(net)


def test_learned_guess_rhs_and_detach(pkg, trained):
    """dg_rhs with the network attached matches the warm-start-free mixed RHS to
    FP32 rounding; detaching restores the previous-pass guesses."""
    om = oracle.Mesh(oracle.MeshSpec(system=1, K=(4, 4, 3), n=6, flux=0, limiter=1, gamma=G))
    gm = pkg.Mesh(system=1, K=(4, 4, 3), n=6, flux=0, limiter=1, gamma=G, precision=1)
    U = om.from_prim(di.blast_sr(om.coords(), seed=3))
    Ro = om.rhs(U)
    gm.set_c2p_net(trained)
    Rl = gm.rhs(_gpu(U)).cpu().numpy()
    gm.set_c2p_net(None)
    Rp = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    sc = np.abs(Ro).max(axis=(0, 2))
    sc = np.maximum(sc, 1e-2 * sc.max())
    el = np.abs(Rl - Ro).max(axis=(0, 2)) / sc
    ep = np.abs(Rp - Ro).max(axis=(0, 2)) / sc
    assert el.max() < 1e-4 and ep.max() < 1e-4, (el, ep)


@pytest.mark.parametrize("n", [7, 8])
def test_learned_guess_more_nodes_than_face_points(pkg, trained, n):
    """n = 7, 8: an element has more nodes than face points, and the guesses of all
    its nodes must fit the face-guess array.  RHS against the oracle at the FP32
    level, and three steps within the 1e-6 bar."""
    om = oracle.Mesh(oracle.MeshSpec(system=1, K=(3, 2, 2), n=n, flux=1, limiter=1, gamma=G))
    gm = pkg.Mesh(system=1, K=(3, 2, 2), n=n, flux=1, limiter=1, gamma=G, precision=1)
    gm.set_c2p_net(trained)
    U = om.from_prim(di.blast_sr(om.coords(), seed=4))
    Ro = om.rhs(U)
    Rl = gm.rhs(_gpu(U)).cpu().numpy()
    assert gm.sync_status() == 0
    sc = np.abs(Ro).max(axis=(0, 2))
    sc = np.maximum(sc, 1e-2 * sc.max())
    assert (np.abs(Rl - Ro).max(axis=(0, 2)) / sc).max() < 1e-4
    Ug = _gpu(U)
    for _ in range(3):
        h = om.cfl_dt(U, 0.2)
        U = om.rk3_step(U, h)
        gm.rk3_step(Ug, dt=h)
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d


def test_learned_guess_cfl_steps_conserve(pkg, trained):
    """CFL-driven steps with the learned guess: device status clean, totals
    conserved to FP32 rounding of the fluxes."""
    om = oracle.Mesh(oracle.MeshSpec(system=1, K=(4, 4, 4), n=4, flux=1, limiter=1, gamma=G))
    gm = pkg.Mesh(system=1, K=(4, 4, 4), n=4, flux=1, limiter=1, gamma=G, precision=1)
    gm.set_c2p_net(trained)
    U = om.from_prim(di.blast_sr(om.coords(), seed=2))
    t0 = om.totals(U)
    Ug = _gpu(U)
    for _ in range(5):
        gm.rk3_step(Ug, cfl=0.2)
    assert gm.sync_status() == 0
    drift = np.abs(om.totals(Ug.cpu().numpy()) - t0) / np.abs(t0).max()
    assert np.all(drift < 1e-7), drift


def test_set_c2p_net_rejects_other_meshes(pkg, trained):
    for system, precision in ((1, 0), (0, 1)):
        m = pkg.Mesh(system=system, K=(2, 2, 2), n=3, flux=1, limiter=0, precision=precision,
                     gamma=G if system else 1.4)
        with pytest.raises(pkg.abi.DGError):
            m.set_c2p_net(trained)
        m.set_c2p_net(None)


def test_full_size_blast_learned_graph_replay(pkg, trained):
    """The bench workload at full size in the bench's launch configuration: the
    mixed path with the learned guess, one CFL step captured into a CUDA graph and
    replayed.  After 10 steps (the oracle takes the GPU's dt sequence) the state
    is within the 1e-6 bar of the FP64 oracle."""
    import torch
    om = oracle.Mesh(oracle.MeshSpec(system=1, K=(16, 16, 16), n=5, flux=1, limiter=1, gamma=G))
    gm = pkg.Mesh(system=1, K=(16, 16, 16), n=5, flux=1, limiter=1, gamma=G, precision=1)
    gm.set_c2p_net(trained)
    U = om.from_prim(di.blast_sr(om.coords(), seed=1))
    Ug = _gpu(U)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt)   # first step (warm-up, outside the graph)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    U = om.rk3_step(U, float(dt.item()))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gm.rk3_step(Ug, cfl=0.2, dt_used=dt)
    for _ in range(9):
        graph.replay()
        torch.cuda.synchronize()
        U = om.rk3_step(U, float(dt.item()))
    assert gm.sync_status() == 0
    d = _rel_l2(om, Ug.cpu().numpy(), U)
    assert np.all(d <= 1e-6), d
