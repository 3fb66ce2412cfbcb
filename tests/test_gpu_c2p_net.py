"""The learned con2prim starting guess: GPU forward and gradient kernels (BF16
tensor cores) against the FP64 CPU reference at the same weights, training on
the GPU, and what the trained guess gains in con2prim iterations."""
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


def _data(seed, n):
    prim = di.c2p_samples(seed, n, gamma=G)
    cons = oracle.prim2con(1, G, prim)
    return cons, prim[4]


def _gpu(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _bf16(x):
    """Round FP32 values to BF16 (nearest even) as numpy float64."""
    import torch
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _params(seed=0):
    p = mlp.init_params(di.uniform(seed, 9, np.arange(mlp.N_PARAMS)))
    p[mlp.OFFSETS["b1"]:mlp.OFFSETS["b1"] + 64] = 0.2 * (di.uniform(seed, 10, np.arange(64)) - 0.5)
    return p.astype(np.float32).astype(np.float64)


def test_forward_matches_cpu_reference(pkg):
    import torch
    cons, p = _data(21, 1000)
    params = _params()
    ref_params = params.copy()
    o = mlp.OFFSETS["W2"]
    ref_params[o:o + 4096] = _bf16(params[o:o + 4096])  # the GPU multiplies BF16 W2
    net = pkg.abi.dg_c2p_net_create(params.astype(np.float32), mlp.DEFAULT_SCALES)
    out = torch.empty(cons.shape[1], dtype=torch.float64, device="cuda")
    pkg.abi.dg_c2p_net_guess(net, cons.shape[1], G, _gpu(cons), out)
    got = out.cpu().numpy()
    ref = mlp.guess(ref_params, cons, G)
    # log-pressure agrees to BF16 rounding of h1 times the output scale
    err = np.abs(np.log10(got) - np.log10(ref))
    assert np.median(err) < 5e-3 and err.max() < 5e-2, (np.median(err), err.max())
    pkg.abi.dg_c2p_net_destroy(net)


def test_gradient_matches_cpu_reference(pkg):
    import torch
    cons, p = _data(22, 1000)
    params = _params(1)
    net = pkg.abi.dg_c2p_net_create(params.astype(np.float32), mlp.DEFAULT_SCALES)
    grad = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    pkg.abi.dg_c2p_net_grad(net, cons.shape[1], _gpu(cons), _gpu(p), grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    ref_params = params.copy()
    o = mlp.OFFSETS["W2"]
    ref_params[o:o + 4096] = _bf16(params[o:o + 4096])
    x, t = mlp.features(cons), mlp.targets(cons, p)
    lref, gref = mlp.loss_and_grad(ref_params, x, t)
    assert abs(loss.item() - lref) <= 2e-2 * lref
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos >= 0.999, cos
    for name, n in (("W1", 192), ("b1", 64), ("W2", 4096), ("b2", 64), ("W3", 64), ("b3", 1)):
        sl = slice(mlp.OFFSETS[name], mlp.OFFSETS[name] + n)
        assert np.linalg.norm(g[sl] - gref[sl]) <= 3e-2 * np.linalg.norm(gref[sl]) + 1e-7, name
    pkg.abi.dg_c2p_net_destroy(net)


def test_training_is_deterministic_and_learns(pkg):
    import torch
    cons, p = _data(23, 1 << 16)
    params = _params(2).astype(np.float32)
    losses = []
    finals = []
    for _ in range(2):
        net = pkg.abi.dg_c2p_net_create(params, mlp.DEFAULT_SCALES)
        lh = torch.zeros(4, dtype=torch.float32, device="cuda")
        pkg.abi.dg_c2p_net_train(net, cons.shape[1], _gpu(cons), _gpu(p), 4, 1024, 3e-3, lh)
        losses.append(lh.cpu().numpy())
        finals.append(pkg.abi.dg_c2p_net_get_params(net))
        pkg.abi.dg_c2p_net_destroy(net)
    assert np.array_equal(finals[0], finals[1]) and np.array_equal(losses[0], losses[1])
    assert np.all(np.diff(losses[0]) < 0) and losses[0][-1] < 0.85 * losses[0][0], losses[0]


def test_learned_guess_cuts_newton_iterations(pkg):
    """Trained on pairs the method generates (a disjoint seed), the network's
    guess leaves con2prim's results unchanged to the solver's own resolution
    while cutting the mean Newton iteration count."""
    import torch
    cons_tr, p_tr = _data(31, 1 << 18)
    net = pkg.abi.dg_c2p_net_create(_params(3).astype(np.float32), mlp.DEFAULT_SCALES)
    pkg.abi.dg_c2p_net_train(net, cons_tr.shape[1], _gpu(cons_tr), _gpu(p_tr), 6, 2048, 2e-3)
    cons, p = _data(32, 100000)
    N = cons.shape[1]
    c = _gpu(cons)
    guess = torch.empty(N, dtype=torch.float64, device="cuda")
    pkg.abi.dg_c2p_net_guess(net, N, G, c, guess)
    outs, its = [], []
    for gs in (None, guess):
        prim = torch.empty((5, N), dtype=torch.float64, device="cuda")
        it = torch.empty(N, dtype=torch.int32, device="cuda")
        st = torch.empty(N, dtype=torch.int32, device="cuda")
        pkg.abi.dg_con2prim(N, G, c, prim, gs, it, st)
        assert int(st.sum().item()) == 0
        outs.append(prim.cpu().numpy())
        its.append(it.cpu().numpy())
    kappa = cons[4] / (p / (G - 1.0))
    rel = np.abs(outs[1][4] - outs[0][4]) / outs[0][4]
    assert np.all(rel <= 4e-15 * (1 + kappa))
    assert its[1].mean() < 0.7 * its[0].mean(), (its[0].mean(), its[1].mean())
    pkg.abi.dg_c2p_net_destroy(net)
