"""GPU tests of the learned warm start: the network's forward pass and
gradient against the FP64 oracle (same bfloat16 weights), training, the cell
features and targets against the oracle's on the same problem, and what the
trained network gains over the plain warm start."""
import numpy as np
import pytest

from oracle import dd as odd
from oracle import mlp as omlp
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    torch.cuda.set_device(0)
    return dd


def _inputs(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, omlp.N_IN)).astype(np.float32)
    X[:, :64] = np.abs(X[:, :64])
    T = rng.normal(size=(n, omlp.N_OUT)).astype(np.float32)
    return X, T


def test_forward_matches_oracle(lib):
    import torch
    params = syn.mlp_init(5)
    X, _ = _inputs(1, 37)
    net = lib.MLP(params)
    y = net.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    net.close()
    ref, _ = omlp.forward(params.astype(np.float64), X.astype(np.float64))
    assert np.abs(y - ref).max() <= 1e-4 * np.abs(ref).max(), np.abs(y - ref).max()


def test_gradient_matches_oracle(lib):
    import torch
    params = syn.mlp_init(6)
    X, T = _inputs(2, 53)
    net = lib.MLP(params)
    loss, g = net.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    net.close()
    loss_ref, g_ref = omlp.backward(params.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in omlp.SHAPES])
    for k, (name, _) in enumerate(omlp.SHAPES):
        a, b = g[offs[k]:offs[k + 1]], g_ref[offs[k]:offs[k + 1]]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-12, name


def test_training_lowers_the_loss(lib):
    import torch
    rng = np.random.default_rng(9)
    X, _ = _inputs(3, 2048)
    A = rng.normal(size=(omlp.N_IN, omlp.N_OUT)).astype(np.float32) / np.sqrt(omlp.N_IN)
    T = np.tanh(X @ A).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    net = lib.MLP(syn.mlp_init(7))
    first = net.train_step(Xd, Td, 1e-3)
    for _ in range(300):
        last = net.train_step(Xd[:512], Td[:512], 1e-3)
    net.close()
    assert last < 0.1 * first, (first, last)


def test_features_and_targets_match_oracle(lib):
    n, b = 32, 4
    mu = syn.gaussian_mixture(n, 3, 40)
    nu = syn.gaussian_mixture(n, 3, 41)
    eps = 2.0 / n ** 2
    sched = [(eps, 3, 0)]
    before = {}

    def keep(prob, part, rows, alpha, e):
        before[part] = list(rows)

    ref = odd.run_schedule(mu, nu, b, 1, sched, odd.Params(err=1e-9), before_half_sweep=keep)
    F_ref, T_ref, _ = omlp.training_pairs(ref.prob, "B", before["B"], ref.alpha["B"], eps)
    g = lib.DD(mu, nu, b, 1, sched, err_tol=1e-7)
    g.run_schedule()
    F, T = g.training_pairs()
    g.close()
    F, T = F.cpu().numpy(), T.cpu().numpy()
    assert F.shape == F_ref.shape and T.shape == T_ref.shape
    assert np.abs(F[:, :64] - F_ref[:, :64]).max() < 1e-5
    assert np.abs(F[:, 64:1088] - F_ref[:, 64:1088]).max() < 1e-3
    assert np.abs(F[:, 1088] - F_ref[:, 1088]).max() < 1e-6
    assert np.abs(T - T_ref).max() < 2e-3, np.abs(T - T_ref).max()


def test_learned_warm_start_gains_over_plain(lib):
    # train on pairs logged from plain runs on other images, then solve new
    # pairs with the plain warm start and with the learned one (compared with
    # the plain one cell by cell): fewer Sinkhorn iterations, same result
    import torch
    from paper_2001_10986_gb300 import learned
    n, b, L = 64, 4, 3
    sched = syn.paper_schedule(n, L, 4)
    Fs, Ts = [], []
    for k in range(4):
        mu = syn.gaussian_mixture(n, 5, 100 + 2 * k)
        nu = syn.gaussian_mixture(n, 5, 101 + 2 * k)
        f, t = learned.log_pairs(mu, nu, b, L, sched, min_level=1)
        Fs.append(f)
        Ts.append(t)
    net = learned.train((torch.cat(Fs), torch.cat(Ts)), epochs=40, batch=256, lr=1e-3)
    # three new pairs; the prediction is compared at the first sweep on each new
    # level. Err = 1e-6 keeps every cell above the FP32 floor of its sums, so
    # that the iteration counts measure the start and not cells that stall
    # there and end in the safeguard
    iters = {0: 0.0, 1: 0.0}
    taken = compared = 0
    costs = {0: [], 1: []}
    for pair in range(3):
        mu = syn.gaussian_mixture(n, 5, 300 + 2 * pair)
        nu = syn.gaussian_mixture(n, 5, 301 + 2 * pair)
        for warm in (0, 1):
            g = lib.DD(mu, nu, b, L, sched, err_tol=1e-6, warm=warm)
            if warm:
                g.attach_mlp(net)
            g.run_schedule()
            p = g.profile()
            iters[warm] += p.sinkhorn_iters
            if warm:
                taken += p.learned_cells
                compared += p.compared_cells
            costs[warm].append(g.cost(with_y=False)[0])
            g.close()
    net.close()
    print("plain iterations %d, learned iterations %d (%d of %d compared cells took the prediction)"
          % (iters[0], iters[1], taken, compared))
    assert compared > 0 and taken > 0
    assert iters[1] < iters[0]
    for c0, c1 in zip(costs[0], costs[1]):
        assert abs(c1 - c0) / c0 < 1e-5
