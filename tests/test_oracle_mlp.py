"""Pins of the learned-warm-start oracle (oracle/mlp.py): bfloat16 rounding,
the network's forward pass on a closed-form case, its gradient against finite
differences, and the features / target definitions against their invariants."""
import numpy as np
import pytest

from oracle import dd as odd
from oracle import mlp
from paper_2001_10986_gb300 import synthetic as syn


def test_bf16_rounding_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even → 1
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, 1 + 2.0 ** -7 + 2.0 ** -8, -2.5, 3.0e38],
                 dtype=np.float32)
    want = [1.0, 1.0, 1 + 2.0 ** -7, 1 + 2.0 ** -6, -2.5, 1.765625 * 2.0 ** 127]
    got = mlp.bf16_round(x)
    np.testing.assert_allclose(got, want, rtol=0, atol=0)
    # bfloat16 keeps 8 significant bits: every result has zero low 16 bits
    assert np.all(got.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


def test_forward_closed_form():
    # W1, W2, W3 select the first 64 inputs; y = relu(x[:64]) + b3
    d = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    for k in range(64):
        d["W1"][k, k] = 1.0
        d["W2"][k, k] = 1.0
        d["W3"][k, k] = 1.0
    d["b3"][:] = np.linspace(-1, 1, 64)
    X = np.random.default_rng(3).normal(size=(5, mlp.N_IN))
    y, _ = mlp.forward(mlp.pack(d), X)
    np.testing.assert_allclose(y, np.maximum(X[:, :64], 0.0) + d["b3"], rtol=0, atol=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    # weights already on the bfloat16 grid, so the rounding does not move them
    params = mlp.bf16_round(syn.mlp_init(11)).astype(np.float64)
    X = rng.normal(size=(3, mlp.N_IN))
    T = rng.normal(size=(3, mlp.N_OUT))
    L, g = mlp.backward(params, X, T)
    # probe biases (exact in FP64) on every layer
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    probe = []
    for k, (name, _) in enumerate(mlp.SHAPES):
        if name.startswith("b"):
            probe += list(rng.choice(np.arange(offs[k], offs[k + 1]), size=6, replace=False))
    h = 1e-6
    for q in probe:
        e = np.zeros_like(params)
        e[q] = h
        fd = (mlp.loss(mlp.forward(params + e, X)[0], T) - mlp.loss(mlp.forward(params - e, X)[0], T)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), (q, fd, g[q])
    # weights: the loss is smooth in a weight away from ReLU kinks, so a step
    # of one bfloat16 ulp on both sides gives the derivative to O(h²)
    for name in ("W1", "W2", "W3"):
        k = [n for n, _ in mlp.SHAPES].index(name)
        for q in rng.choice(np.arange(offs[k], offs[k + 1]), size=4, replace=False):
            w = params[q]
            ulp = 2.0 ** (np.floor(np.log2(abs(w))) - 7) if w != 0 else 2.0 ** -40
            e = np.zeros_like(params)
            e[q] = ulp
            fd = (mlp.loss(mlp.forward(params + e, X)[0], T) - mlp.loss(mlp.forward(params - e, X)[0], T)) / (2 * ulp)
            assert abs(fd - g[q]) <= 1e-3 * max(1e-6, abs(g[q])) + 1e-9, (name, q, fd, g[q])


@pytest.fixture(scope="module")
def small_grid():
    n, b = 32, 4
    mu = syn.gaussian_mixture(n, 3, 20)
    nu = syn.gaussian_mixture(n, 3, 21)
    return odd.GridProblem(mu, nu, b, 1.0 / n)


def test_features_normalised_and_windowed(small_grid):
    prob = small_grid
    J = prob.parts["A"][5]
    # ν_cell = one point mass: the histogram is 1024 at the window centre
    y = 17 * prob.n + 9
    f = mlp.cell_features(prob, J, np.array([y]), np.array([0.3]), 2.0 / prob.n ** 2)
    assert abs(f[:64].mean() - 1.0) < 1e-12
    hist = f[64:1088].reshape(32, 32)
    assert hist[16, 16] == 1024.0 and hist.sum() == 1024.0
    assert abs(f[1088] - np.log(2.0)) < 1e-12


def test_target_removes_the_translation_of_nu(small_grid):
    # the converged α of a cell for ν_cell and for ν_cell moved by an integer
    # offset differ by the linear term −2⟨x,t⟩ (+ const): equal targets
    prob = small_grid
    J = prob.parts["A"][9]
    X = np.sort(prob.cell_points(J))
    eps = 2.0 / prob.n ** 2
    cols = np.arange(prob.n * prob.n)
    yr, yc = np.divmod(cols, prob.n)
    base = np.exp(-((yr - 14.3) ** 2 + (yc - 11.7) ** 2) / 18.0)
    keep = (yr < 26) & (yc < 26) & (yr > 2) & (yc > 2)
    targets, checks = [], []
    for (tr, tc) in [(0, 0), (3, -2)]:
        sel = cols[keep] + tr * prob.n + tc
        nu_cell = base[keep] * prob.mu[X].sum() / base[keep].sum()
        C = prob.cost(X, sel)
        f0 = eps * np.log(prob.mu[X])
        f, g, P, it, err = odd.sinkhorn_cell(C, prob.mu[X], nu_cell, f0, eps, 1e-12, 20000)
        alpha = np.zeros(prob.mu.size)
        alpha[X] = f - eps * np.log(prob.mu[X])
        anc = mlp.anchor(prob, J, sel, nu_cell)
        targets.append(mlp.cell_target(prob, J, alpha, eps, anc))
        # the prediction of the exact target maps back to α up to a constant
        checks.append(np.ptp(mlp.alpha_from_prediction(prob, J, targets[-1], eps, anc) - alpha[X]) / eps)
    assert abs(targets[0].mean()) < 1e-12
    np.testing.assert_allclose(targets[0], targets[1], rtol=0, atol=1e-6)
    assert max(checks) < 1e-9
