"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what it pins. None of them compares the oracle with itself:
the references are an independent full-problem Sinkhorn (scaling form), an LP
solver, the rate bound of Theorem 4.1, the odd-even transposition sort of §5,
the identities of Lemmas 4.2/4.3, Proposition 2.5 and Proposition 6.1, and
closed forms.
"""
import json
import os

import numpy as np
import pytest

from oracle import dd, referees
from paper_2001_10986_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(n, b, blobs, seed):
    mu = syn.gaussian_mixture(n, blobs, 2 * seed)
    nu = syn.gaussian_mixture(n, blobs, 2 * seed + 1)
    return dd.GridProblem(mu, nu, b, 1.0 / n)


def _full_cost(prob):
    return prob.cost(np.arange(prob.mu.size), np.arange(prob.nu.size))


# --------------------------------------------------------------------------
# cell solver: one composite cell covering X is plain Sinkhorn (textbook)
# --------------------------------------------------------------------------
def test_single_cell_is_plain_sinkhorn():
    prob = _grid(8, 4, 2, 0)           # 2×2 basic cells: partition A = one cell
    eps = 0.02
    alpha = np.zeros(64)
    rows, info = dd.half_sweep(prob, "A", dd.product_state(prob), alpha, eps,
                               dd.Params(err=1e-12, trunc=0.0))
    P = dd.partition_plan(prob, "A", rows, alpha, eps)
    Pr, _, _ = referees.sinkhorn_scaling(prob.mu, prob.nu, _full_cost(prob), eps)
    assert np.abs(P - Pr).sum() / Pr.sum() < 1e-9
    # the stored marginals are the row sums of that plan over each basic cell
    for i, X in enumerate(prob.basic):
        c, v = rows[i]
        np.testing.assert_allclose(v, Pr[X][:, c].sum(axis=0), rtol=1e-8, atol=1e-13)


def test_sinkhorn_cell_ends_on_y_iteration():
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, (5, 7))
    mu = rng.uniform(0.5, 1, 5); mu /= mu.sum()
    nu = rng.uniform(0.5, 1, 7); nu /= nu.sum()
    f, g, P, it, ex = dd.sinkhorn_cell(C, mu, nu, np.zeros(5), 0.1, 1e-3, 3)
    np.testing.assert_allclose(P.sum(axis=0), nu, rtol=1e-13)       # Y exact
    assert ex == pytest.approx(np.abs(P.sum(axis=1) - mu).sum(), rel=1e-12)


# --------------------------------------------------------------------------
# global optimality: converged DD at fixed ε equals the full Sinkhorn solution
# --------------------------------------------------------------------------
def test_converged_dd_equals_global_sinkhorn():
    prob = _grid(8, 2, 2, 1)            # 4×4 basic cells, 4 A cells, 9 B cells
    eps = 0.03
    Pr, _, _ = referees.sinkhorn_scaling(prob.mu, prob.nu, _full_cost(prob), eps)
    rows = dd.product_state(prob)
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    par = dd.Params(err=1e-12, trunc=0.0, max_iter=5000)
    for _ in range(60):
        for part in "AB":
            rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
    P = dd.partition_plan(prob, "B", rows, alpha["B"], eps)
    assert np.abs(P - Pr).sum() / Pr.sum() < 1e-8


def test_converged_dd_with_massless_pixels_equals_global_sinkhorn():
    # pixels without mass in μ and in ν: the cells are solved on the support
    # of μ_J, and the converged decomposition still equals the global
    # scaling-form Sinkhorn (which gives those rows and columns zero mass)
    prob = _grid(8, 2, 2, 1)
    mu, nu = prob.mu.copy(), prob.nu.copy()
    mu[[5, 18, 41]] = 0.0
    nu[[0, 27, 63]] = 0.0
    mu /= mu.sum()
    nu /= nu.sum()
    prob = dd.GridProblem(mu.reshape(8, 8), nu.reshape(8, 8), 2, 1.0 / 8)
    eps = 0.03
    Pr, _, _ = referees.sinkhorn_scaling(prob.mu, prob.nu, _full_cost(prob), eps)
    rows = dd.product_state(prob)
    rows = [(c[v > 0], v[v > 0]) for c, v in rows]
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    par = dd.Params(err=1e-12, trunc=0.0, max_iter=5000)
    with np.errstate(divide="ignore"):
        for _ in range(60):
            for part in "AB":
                rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
        P = dd.partition_plan(prob, "B", rows, alpha["B"], eps)
    assert np.all(np.isfinite(alpha["A"])) and np.all(np.isfinite(alpha["B"]))
    assert np.abs(P - Pr).sum() / Pr.sum() < 1e-8
    assert P[[5, 18, 41]].sum() == 0.0 and P[:, [0, 27, 63]].sum() == 0.0


# --------------------------------------------------------------------------
# ε → 0: entropic cost is within ε·min(H(μ),H(ν)) above the LP optimum
# --------------------------------------------------------------------------
def test_small_eps_against_lp():
    prob = _grid(8, 2, 2, 2)            # 64 pixels
    C = _full_cost(prob)
    lp_cost, _ = referees.lp_optimum(prob.mu, prob.nu, C)
    H = min(-(prob.mu * np.log(prob.mu)).sum(), -(prob.nu * np.log(prob.nu)).sum())
    rows = dd.product_state(prob)
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    par = dd.Params(err=1e-10, trunc=0.0, max_iter=20000)
    for eps, sweeps, _ in syn.halving_schedule(0.05, 0.05 / 16, 20):
        for _ in range(sweeps):
            for part in "AB":
                rows, info = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
        cost = info.cost
        # ⟨c, π_ε⟩ ≥ C* by feasibility; ⟨c, π_ε⟩ − C* ≤ ε·KL(π_0|μ⊗ν) ≤ ε·H
        assert cost >= lp_cost - 1e-9
        assert cost - lp_cost <= eps * H * (1 + 1e-6) + 1e-9


# --------------------------------------------------------------------------
# worst-case examples of §4.3 (golden setups from Fig. WorstCaseSetup)
# --------------------------------------------------------------------------
def _three_cell_deltas(eps, q, n_iter):
    g = json.load(open(os.path.join(GOLDEN, "three_cell_worst_case.json")))
    C = np.array(g["cost"], dtype=float)
    p = (1 - q) / 2
    mu = np.array([p, q, p]); nu = mu.copy()
    prob = dd.matrix_problem(mu, nu, C, [[0], [1], [2]],
                             {"A": [[0, 1], [2]], "B": [[0], [1, 2]]})
    # π⁰ = p·δ(1,3) + q·δ(2,2) + p·δ(3,1)
    rows = [(np.array([2]), np.array([p])), (np.array([1]), np.array([q])),
            (np.array([0]), np.array([p]))]
    alpha = {"A": np.zeros(3), "B": np.zeros(3)}
    Pr, _, _ = referees.sinkhorn_scaling(mu, nu, C, eps, tol=1e-15)
    kl_star = dd.kl_minus_mass(Pr, C, mu, nu, eps)
    par = dd.Params(err=1e-14, trunc=0.0, max_iter=100000)
    D = []
    for l in range(n_iter):
        part = "AB"[l % 2]
        rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
        P = dd.partition_plan(prob, part, rows, alpha[part], eps)
        D.append(dd.kl_minus_mass(P, C, mu, nu, eps) - kl_star)
    return np.array(D), float(g["cost_sup_norm"])


@pytest.mark.parametrize("eps", [3.0, 5.0, 10.0, 20.0])
def test_three_cell_rate_bound_eps(eps):
    q = 0.3
    D, cn = _three_cell_deltas(eps, q, 40)
    bound = 1.0 / (1.0 + np.exp(-2 * cn / eps) * q / (1 - q))   # eq. LambdaBound
    ok = D[:-1] > 1e-11
    lam = D[1:][ok] / D[:-1][ok]
    assert lam.size >= 3
    assert np.all(D[1:][ok] >= -1e-12)
    assert np.all(lam <= bound * (1 + 1e-9))


@pytest.mark.parametrize("q", [0.1, 0.3, 0.5])
def test_three_cell_rate_bound_q(q):
    eps = 10.0                                                   # Example 4.11
    D, cn = _three_cell_deltas(eps, q, 40)
    ok = D[:-1] > 1e-11
    lam = D[1:][ok] / D[:-1][ok]
    # eq. LambdaBoundQ: λ(q)⁻¹ − 1 ≥ e^{−2‖c‖/ε}·q/(1−q)
    assert np.all(1.0 / lam - 1.0 >= np.exp(-2 * cn / eps) * q / (1 - q) * (1 - 1e-9))


def test_three_cell_rate_slows_with_smaller_eps():
    lam = []
    for eps in (2.0, 4.0, 8.0):
        D, _ = _three_cell_deltas(eps, 0.3, 40)
        ok = D[:-1] > 1e-11
        lam.append(np.median(D[1:][ok] / D[:-1][ok]))
    assert lam[0] > lam[1] > lam[2]


def test_chain_rate_increases_with_n():
    g = json.load(open(os.path.join(GOLDEN, "chain_worst_case.json")))
    eps = g["eps"]
    lams = []
    for N in (4, 6, 8):
        C = np.full((N, N), float(g["cost_other"]))
        np.fill_diagonal(C, g["cost_diag"])
        C[0, N - 1] = C[N - 1, 0] = g["cost_corner"]
        mu = np.full(N, 1.0 / N); nu = mu.copy()
        A = [[k, k + 1] for k in range(0, N, 2)]
        B = [[0]] + [[k, k + 1] for k in range(1, N - 1, 2)] + [[N - 1]]
        prob = dd.matrix_problem(mu, nu, C, [[k] for k in range(N)], {"A": A, "B": B})
        sigma = list(range(N)); sigma[0], sigma[N - 1] = N - 1, 0
        rows = [(np.array([sigma[k]]), np.array([1.0 / N])) for k in range(N)]
        alpha = {"A": np.zeros(N), "B": np.zeros(N)}
        Pr, _, _ = referees.sinkhorn_scaling(mu, nu, C, eps, tol=1e-15)
        kls = dd.kl_minus_mass(Pr, C, mu, nu, eps)
        par = dd.Params(err=1e-12, trunc=0.0, max_iter=2000)
        D = []
        for l in range(60):
            part = "AB"[l % 2]
            rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
            P = dd.partition_plan(prob, part, rows, alpha[part], eps)
            D.append(dd.kl_minus_mass(P, C, mu, nu, eps) - kls)
        D = np.array(D)
        ok = D[:-2] > 1e-10
        lams.append(np.median((D[2:][ok] / D[:-2][ok])))   # per A+B sweep
    assert lams[0] < lams[1] < lams[2] < 1.0


# --------------------------------------------------------------------------
# §5: small-ε DD with singleton cells and a Monge cost is odd-even sorting
# --------------------------------------------------------------------------
def test_odd_even_transposition_sort():
    N = 8
    x = np.arange(N, dtype=float)
    C = (x[:, None] - x[None, :]) ** 2          # strictly Monge
    mu = np.full(N, 1.0 / N); nu = mu.copy()
    A = [[k, k + 1] for k in range(0, N, 2)]
    B = [[0]] + [[k, k + 1] for k in range(1, N - 1, 2)] + [[N - 1]]
    prob = dd.matrix_problem(mu, nu, C, [[k] for k in range(N)], {"A": A, "B": B})
    perm = np.array([5, 2, 7, 0, 6, 1, 4, 3])
    rows = [(np.array([perm[k]]), np.array([1.0 / N])) for k in range(N)]
    alpha = {"A": np.zeros(N), "B": np.zeros(N)}
    expect = referees.odd_even_transposition_sort_steps(perm, N)
    par = dd.Params(err=1e-12, trunc=1e-15, max_iter=1000)
    for step in range(N):
        part = "AB"[step % 2]
        rows, _ = dd.half_sweep(prob, part, rows, alpha[part], 0.05, par)
        got = np.array([c[np.argmax(v)] for c, v in rows])
        np.testing.assert_array_equal(got, expect[step])
    np.testing.assert_array_equal(got, np.arange(N))


# --------------------------------------------------------------------------
# invariants: feasibility (Prop. 3.2), Balance, refinement (Prop. 6.1)
# --------------------------------------------------------------------------
def test_invariants_multiscale_run():
    mu = syn.gaussian_mixture(16, 3, 4)
    nu = syn.gaussian_mixture(16, 3, 5)
    sched = syn.paper_schedule(16, 2, 3)
    par = dd.Params(err=1e-8)
    checks = []

    def check(prob, part, rows, alpha, eps, info):
        s = np.zeros(prob.nu.size)
        for c, v in rows:
            assert np.all(v > 0)
            assert np.all(np.diff(c) > 0)
            np.add.at(s, c, v)
        # Σ_i ν_i = ν up to rounding and the mass dropped by Truncate
        assert np.abs(s - prob.nu).sum() <= info.truncated_mass + 1e-12
        m = np.array([v.sum() for _, v in rows])
        assert np.abs(m - prob.basic_mass).max() <= info.truncated_mass + 1e-13
        checks.append(info.err_x)

    res = dd.run_schedule(mu, nu, 2, 2, sched, par, on_half_sweep=check)
    assert len(checks) == 2 * sum(s for _, s, _ in sched)
    assert res.prob.n == 16


def test_balance_measures_invariants():
    rng = np.random.default_rng(0)
    parts = [rng.uniform(0, 1, 20) for _ in range(4)]
    total = sum(parts)
    targets = np.array([p.sum() for p in parts]) + np.array([0.3, -0.1, -0.25, 0.05])
    out = dd.balance_measures([p.copy() for p in parts], targets)
    np.testing.assert_allclose(sum(out), total, rtol=1e-14)
    np.testing.assert_allclose([p.sum() for p in out], targets, rtol=1e-13)
    assert all(np.all(p >= 0) for p in out)
    # no-op when masses already match
    out2 = dd.balance_measures([p.copy() for p in parts], [p.sum() for p in parts])
    for a, b in zip(out2, parts):
        np.testing.assert_array_equal(a, b)


def test_refined_marginals_are_feasible():
    mus = dd.pyramid(syn.gaussian_mixture(16, 3, 6), 2)
    nus = dd.pyramid(syn.gaussian_mixture(16, 3, 7), 2)
    coarse = dd.GridProblem(mus[0], nus[0], 2, 1 / 8)
    fine = dd.GridProblem(mus[1], nus[1], 2, 1 / 16)
    rows = dd.product_state(coarse)
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    par = dd.Params(err=1e-8)
    for part in "AB":
        rows, _ = dd.half_sweep(coarse, part, rows, alpha[part], 0.05, par)
    rows_f = dd.refine_basic_marginals(coarse, fine, rows)
    s = np.zeros(256)
    for c, v in rows_f:
        np.add.at(s, c, v)
    np.testing.assert_allclose(s, fine.nu, rtol=1e-12, atol=1e-17)       # Σ_i ν_i⁰ = ν
    np.testing.assert_allclose([v.sum() for _, v in rows_f], fine.basic_mass, rtol=1e-12)


def test_pyramid_is_push_forward():
    img = syn.gaussian_mixture(16, 2, 9)
    p = dd.pyramid(img, 3)
    assert [a.shape[0] for a in p] == [4, 8, 16]
    assert p[0][1, 2] == pytest.approx(img[4:8, 8:12].sum(), rel=1e-14)


def test_refined_duals_reproduce_linear_and_quadratic_terms():
    # α linear in the pixel position must be refined exactly (first order),
    # whatever the cell; positions in coarse pixel units, fine pixels at ±¼.
    mus = dd.pyramid(syn.gaussian_mixture(16, 2, 10), 2)
    coarse = dd.GridProblem(mus[0], mus[0], 2, 1 / 8)
    fine = dd.GridProblem(mus[1], mus[1], 2, 1 / 16)
    pi, pj = np.divmod(np.arange(64), 8)
    a_c = 0.7 * pi - 1.3 * pj + 0.25
    for part in "AB":
        a_f = dd.refine_duals(coarse, fine, a_c, part)
        fi, fj = np.divmod(np.arange(256), 16)
        expect = 0.7 * ((fi + 0.5) / 2 - 0.5) - 1.3 * ((fj + 0.5) / 2 - 0.5) + 0.25
        np.testing.assert_allclose(a_f, expect, atol=1e-13)


# --------------------------------------------------------------------------
# objective: monotone decrease and the decrement identity (Lemma 4.3),
# the scaling formula (Lemma 4.2), weak duality (Prop. 2.5)
# --------------------------------------------------------------------------
def test_kl_monotone_and_decrement_identity():
    prob = _grid(8, 2, 2, 11)
    eps = 0.04
    C = _full_cost(prob)
    rows = dd.product_state(prob)
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    par = dd.Params(err=1e-13, trunc=0.0, max_iter=20000)
    prev, prev_kl = None, None
    for l in range(8):
        part = "AB"[l % 2]
        rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
        P = dd.partition_plan(prob, part, rows, alpha[part], eps)
        kl = dd.kl_minus_mass(P, C, prob.mu, prob.nu, eps)
        if prev is not None:
            assert kl <= prev_kl + 1e-12
            dec = dd.kl_div(prev, P)
            assert prev_kl - kl == pytest.approx(dec, rel=1e-6, abs=1e-12)
        prev, prev_kl = P, kl


def test_lemma_4_2_scaling_formula():
    prob = _grid(8, 2, 2, 12)
    eps = 0.05
    C = _full_cost(prob)
    rows = dd.product_state(prob)
    alpha = {"A": np.zeros(64), "B": np.zeros(64)}
    plans = {}
    par = dd.Params(err=1e-12, trunc=0.0)
    rows, _ = dd.half_sweep(prob, "A", rows, alpha["A"], eps, par)
    rows, _ = dd.half_sweep(prob, "B", rows, alpha["B"], eps, par, plans=plans)
    P = np.zeros((64, 64))
    lhs_sum = 0.0
    for X, cols, Pc in plans.values():
        P[np.ix_(X, cols)] = Pc
        # dπ_J/dK = u(x)·v(y); log u = α/ε; log v from the cell's Y-iteration
        f = alpha["B"][X] + eps * np.log(prob.mu[X])
        Cc = C[np.ix_(X, cols)]
        nu_c = Pc.sum(axis=0)
        g = eps * np.log(nu_c) - eps * dd.logsumexp((f[:, None] - Cc) / eps, axis=0)
        logu = alpha["B"][X] / eps
        logv = (g - eps * np.log(prob.nu[cols])) / eps
        lhs_sum += Pc.sum(axis=1) @ logu + Pc.sum(axis=0) @ logv
    K = dd.kernel_mass(C, prob.mu, prob.nu, eps)
    direct = dd.kl_minus_mass(P, C, prob.mu, prob.nu, eps) + K
    lemma = lhs_sum - P.sum() + K
    assert direct == pytest.approx(lemma, rel=1e-10)


def test_weak_duality_and_zero_gap_at_optimum():
    prob = _grid(8, 4, 2, 13)
    eps = 0.05
    C = _full_cost(prob)
    Pr, u, v = referees.sinkhorn_scaling(prob.mu, prob.nu, C, eps, tol=1e-15)
    K = dd.kernel_mass(C, prob.mu, prob.nu, eps)
    primal = dd.kl_minus_mass(Pr, C, prob.mu, prob.nu, eps) + K
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = rng.normal(0, eps, 64); b = rng.normal(0, eps, 64)
        assert dd.dual_objective(a, b, prob.mu, prob.nu, C, prob.mu, prob.nu, eps) <= primal + 1e-12
    J = dd.dual_objective(eps * np.log(u), eps * np.log(v), prob.mu, prob.nu, C, prob.mu, prob.nu, eps)
    assert J == pytest.approx(primal, rel=1e-10)


def test_partitions_cover_and_graph_connected():
    nb = 6
    parts = dd.grid_partitions(nb)
    for name in "AB":
        flat = sorted(i for J in parts[name] for i in J)
        assert flat == list(range(nb * nb))
    assert len(parts["A"]) == 9 and len(parts["B"]) == 16
    assert sum(len(J) == 1 for J in parts["B"]) == 4
    # partition graph (Def. 4.5): basic cells joined when they share a cell
    adj = {i: set() for i in range(nb * nb)}
    for name in "AB":
        for J in parts[name]:
            for i in J:
                adj[i].update(J)
    seen, todo = {0}, [0]
    while todo:
        k = todo.pop()
        for m in adj[k] - seen:
            seen.add(m); todo.append(m)
    assert len(seen) == nb * nb


# --------------------------------------------------------------------------
# cell-by-cell objective (§6.3) and the cell problems' primal-dual gaps
# --------------------------------------------------------------------------
def _state_after(prob, eps, sweeps, err, max_iter=20000, trunc=0.0):
    rows = dd.product_state(prob)
    alpha = {"A": np.zeros(prob.mu.size), "B": np.zeros(prob.mu.size)}
    par = dd.Params(err=err, trunc=trunc, max_iter=max_iter)
    for l in range(2 * sweeps):
        part = "AB"[l % 2]
        rows, _ = dd.half_sweep(prob, part, rows, alpha[part], eps, par)
    return rows, alpha


def test_cell_primals_sum_to_kl_of_the_partition_plan():
    prob = _grid(16, 4, 3, 14)
    eps = 0.01
    rows, alpha = _state_after(prob, eps, 2, 1e-6)
    primal, _ = dd.cell_objectives(prob, "B", rows, alpha["B"], eps)
    P = dd.partition_plan(prob, "B", rows, alpha["B"], eps)
    kl = dd.kl_minus_mass(P, _full_cost(prob), prob.mu, prob.nu, eps)
    assert primal.sum() == pytest.approx(kl, rel=1e-12)


def test_cell_gap_is_the_marginal_residual_form():
    # π_J = u ⊗ v · K: the gap KL(π_J|K_J) − J_J(u, v) equals
    # ⟨P_X π_J − μ_J, log u⟩ + ⟨P_Y π_J − ν_cell, log v⟩ (Lemma 4.2 on the
    # cell); log v is read off the plan itself, not from the oracle's β
    prob = _grid(16, 4, 3, 15)
    eps = 0.01
    rows, alpha = _state_after(prob, eps, 1, 1e-6, max_iter=3)
    primal, gap = dd.cell_objectives(prob, "B", rows, alpha["B"], eps)
    assert np.abs(gap).max() > 1e-6          # an unconverged state has a gap
    for j, J in enumerate(prob.parts["B"]):
        cols, nu_cell = dd.gather(rows, J)
        X = prob.cell_points(J)
        C = prob.cost(X, cols)
        f = alpha["B"][X] + eps * np.log(prob.mu[X])
        g = eps * np.log(nu_cell) - eps * dd.logsumexp((f[:, None] - C) / eps, axis=0)
        P = np.exp((f[:, None] + g[None, :] - C) / eps)
        logK = -C / eps + np.log(prob.mu[X])[:, None] + np.log(prob.nu[cols])[None, :]
        logu = alpha["B"][X] / eps
        logv = (np.log(P) - logK - logu[:, None]).mean(axis=0)
        res = (P.sum(1) - prob.mu[X]) @ logu + (P.sum(0) - nu_cell) @ logv
        assert gap[j] == pytest.approx(res, rel=1e-8, abs=1e-14)
        lemma = P.sum(1) @ logu + P.sum(0) @ logv - P.sum()
        assert primal[j] == pytest.approx(lemma, rel=1e-10)


def test_cell_gap_vanishes_at_the_optimum_and_ignores_cell_constants():
    prob = _grid(16, 4, 3, 16)
    eps = 0.01
    rows, alpha = _state_after(prob, eps, 2, 1e-13)
    primal, gap = dd.cell_objectives(prob, "B", rows, alpha["B"], eps)
    assert np.abs(gap).max() < 1e-10 * np.abs(primal).sum()
    # a constant added to α on one cell moves β by the opposite constant:
    # the gap changes by c/ε·(‖ν_cell‖ − ‖μ_J‖), which is zero here (no
    # truncation, BalanceMeasures makes the masses equal)
    rows2, alpha2 = _state_after(prob, eps, 1, 1e-6, max_iter=3)
    _, g0 = dd.cell_objectives(prob, "B", rows2, alpha2["B"], eps)
    shifted = alpha2["B"].copy()
    shifted[prob.cell_points(prob.parts["B"][3])] += 7.0 * eps
    _, g1 = dd.cell_objectives(prob, "B", rows2, shifted, eps)
    assert g1 == pytest.approx(g0, rel=1e-9, abs=1e-13)


# --------------------------------------------------------------------------
# dual gluing (§6.3), eq. RelPDGap, glued dual refinement (§6.4)
# --------------------------------------------------------------------------
def test_gluing_graph_connects_the_a_cells():
    prob = _grid(16, 2, 2, 20)            # 8×8 basic cells: 4×4 A cells, 5×5 B cells
    edges = dd.gluing_graph(prob)
    nA = len(prob.parts["A"])
    seen = {0}
    frontier = [0]
    while frontier:
        j = frontier.pop()
        for j1, j2, *_ in edges:
            if j1 == j and j2 not in seen:
                seen.add(j2)
                frontier.append(j2)
    assert seen == set(range(nA))
    for j1, j2, jb, X1, X2 in edges:       # X1, X2 lie in J1 ∩ J_B and J2 ∩ J_B
        assert set(X1) <= set(prob.cell_points(prob.parts["A"][j1]))
        assert set(X1) <= set(prob.cell_points(prob.parts["B"][jb]))
        assert set(X2) <= set(prob.cell_points(prob.parts["A"][j2]))
        assert (j2, j1, jb) in {(a, b, c) for a, b, c, *_ in edges}


def test_glued_duals_of_consistent_rescalings_are_one_dual():
    # u_{A,J} = λ_J u*, u_{B,J} = κ_J u*: the glued û is a constant multiple
    # of u* (the path-product construction of §6.3); the sign of log q in the
    # least-squares problem decides this (the opposite sign gives λ_J² u*)
    prob = _grid(16, 2, 2, 21)
    eps = 0.02
    rng = np.random.default_rng(5)
    a_star = eps * rng.normal(0.0, 2.0, prob.mu.size)
    aA, aB = a_star.copy(), a_star.copy()
    for J in prob.parts["A"]:
        aA[prob.cell_points(J)] += eps * rng.normal(0.0, 3.0)
    for J in prob.parts["B"]:
        aB[prob.cell_points(J)] += eps * rng.normal(0.0, 3.0)
    a_hat, _ = dd.glue_duals(prob, aA, aB, eps)
    assert np.ptp(a_hat - a_star) / eps < 1e-9


def test_glued_duals_at_convergence_close_the_gap():
    # converged DD = global Sinkhorn: the glued duals are the global scaling
    # up to a constant and eq. RelPDGap vanishes
    prob = _grid(16, 4, 3, 22)
    eps = 0.02
    rows, alpha = _state_after(prob, eps, 40, 1e-13)
    a_hat, _ = dd.glue_duals(prob, alpha["A"], alpha["B"], eps)
    C = _full_cost(prob)
    _, u, _ = referees.sinkhorn_scaling(prob.mu, prob.nu, C, eps, tol=1e-14)
    assert np.ptp(a_hat - eps * np.log(u)) / eps < 1e-6
    b_hat = dd.best_y_dual(prob, a_hat, eps)
    P = dd.partition_plan(prob, "B", rows, alpha["B"], eps)
    rel, gap, primal = dd.relative_pd_gap(prob, P, a_hat, b_hat, eps)
    assert abs(rel) < 1e-8


def test_glued_duals_keep_weak_duality_before_convergence():
    # Prop. 2.5 (ii): J(û, v̂) ≤ KL(π|K) for every coupling π of μ and ν, here
    # the optimal one and the product μ⊗ν, with the glued duals of an
    # unconverged state; the gap is strictly positive there
    prob = _grid(16, 4, 3, 23)
    eps = 0.02
    rows, alpha = _state_after(prob, eps, 1, 1e-6, max_iter=3)
    a_hat, _ = dd.glue_duals(prob, alpha["A"], alpha["B"], eps)
    b_hat = dd.best_y_dual(prob, a_hat, eps)
    C = _full_cost(prob)
    Pstar, _, _ = referees.sinkhorn_scaling(prob.mu, prob.nu, C, eps, tol=1e-14)
    _, gap_star, _ = dd.relative_pd_gap(prob, Pstar, a_hat, b_hat, eps)
    _, gap_prod, _ = dd.relative_pd_gap(prob, np.outer(prob.mu, prob.nu), a_hat, b_hat, eps)
    assert gap_star > 1e-8
    assert gap_prod > gap_star


def test_glued_refinement_interpolates_linearly():
    # fine pixel I sits at t = I/2 − 1/4 in coarse index units: an affine α̂
    # is reproduced exactly, and α̂ = k² becomes t² + w(1 − w) with
    # w ∈ {1/4, 3/4} inside (3/16) and w ∈ {−1/4, 5/4} at the two borders (−5/16)
    coarse = _grid(8, 2, 2, 24)
    fine = _grid(16, 2, 2, 25)
    k = np.arange(8.0)
    t = np.arange(16) / 2.0 - 0.25
    aff = (0.3 + 0.7 * k[:, None] - 1.1 * k[None, :]).ravel()
    got = dd.refine_duals_glued(coarse, fine, aff).reshape(16, 16)
    assert np.allclose(got, 0.3 + 0.7 * t[:, None] - 1.1 * t[None, :], rtol=0, atol=1e-12)
    quad = np.repeat((k ** 2)[:, None], 8, axis=1).ravel()
    got = dd.refine_duals_glued(coarse, fine, quad).reshape(16, 16)[:, 5]
    want = t ** 2 + 3.0 / 16.0
    want[[0, -1]] = t[[0, -1]] ** 2 - 5.0 / 16.0
    assert np.allclose(got, want, rtol=0, atol=1e-12)


def test_glued_refinement_reaches_the_same_fixed_point():
    mu = syn.gaussian_mixture(16, 3, 60)
    nu = syn.gaussian_mixture(16, 3, 61)
    sched = [(0.02, 3, 0), (0.01, 25, 1)]
    par = dd.Params(err=1e-12, trunc=0.0)
    r_cell = dd.run_schedule(mu, nu, 4, 2, sched, par)
    a = dd.rows_to_dense(r_cell.rows, 256)
    for mode in ("glued", "hybrid"):
        r = dd.run_schedule(mu, nu, 4, 2, sched, par, dual_refinement=mode)
        assert np.abs(a - dd.rows_to_dense(r.rows, 256)).sum() < 1e-8, mode


def test_table1_protocol_magnitudes_at_64():
    # the paper's protocol on a 64² pair of synthetic mixtures: magnitudes of
    # Table 1's 64×64 column (its images are not available, so the bands are
    # wide): relative PD gap with glued duals (eq. RelPDGap), marginal errors
    # within the stopping criterion, entries per pixel at the largest ε of the
    # finest layer and at the end
    with open(os.path.join(GOLDEN, "table1_64.json")) as f:
        ref = json.load(f)
    n = 64
    sched, levels = syn.table1_schedule(n)
    assert 2 * sum(s for _, s, _ in sched) == (6 - 2) * 8 + 2
    mu = syn.gaussian_mixture(n, 6, 0, floor=1e-4)
    nu = syn.gaussian_mixture(n, 6, 1, floor=1e-4)
    nnz = []

    def count(prob, part, rows, alpha, eps, info):
        if prob.n == n:
            nnz.append(sum(r[0].size for r in rows))

    r = dd.run_schedule(mu, nu, 4, levels, sched, dd.Params(err=ref["err"]), on_half_sweep=count)
    prob = r.prob
    a_hat, _ = dd.glue_duals(prob, r.alpha["A"], r.alpha["B"], r.eps)
    b_hat = dd.best_y_dual(prob, a_hat, r.eps)
    P = dd.partition_plan(prob, r.last_part, r.rows, r.alpha[r.last_part], r.eps)
    rel, _, _ = dd.relative_pd_gap(prob, P, a_hat, b_hat, r.eps)
    err_x = np.abs(P.sum(axis=1) - prob.mu).sum()
    err_y = dd.y_marginal_error(prob, r.rows)
    assert 0.0 < rel < 10 * ref["relative_pd_gap"][0]
    assert err_x <= ref["err"]
    assert err_y < ref["l1_marginal_error_y"][0] + ref["l1_marginal_error_y"][1]
    per_px_max = ref["entries_max"][0] / ref["pixels"]
    per_px_final = ref["entries_final"][0] / ref["pixels"]
    assert 0.5 * per_px_max < max(nnz) / n**2 < 2.0 * per_px_max
    assert 0.4 * per_px_final < nnz[-1] / n**2 < 2.5 * per_px_final


def test_helmholtz_potential_of_an_exact_gradient():
    # log q(j1, j2) = φ(j2) − φ(j1) on a cycle with both orientations: the
    # least-squares potential is φ up to its mean (closed form)
    j1 = np.array([0, 1, 2, 3, 1, 2, 3, 0])
    j2 = np.array([1, 2, 3, 0, 0, 1, 2, 3])
    phi = np.array([0.3, -1.2, 2.5, 0.1])
    V = dd.helmholtz_potential(4, j1, j2, phi[j2] - phi[j1])
    assert np.allclose(V, phi - phi.mean(), atol=1e-12)


def test_stop_rule_after_truncation_loss():
    # ν_cell lighter than μ_J by δ (mass that Truncate removed): no coupling
    # of the cell meets μ_J, and the rescaled stop rule still ends the solve;
    # at its end P_X π = μ·‖ν‖/‖μ‖ up to the tolerance, so the reported
    # (unscaled) X-error is δ in closed form
    rng = np.random.default_rng(7)
    C = rng.uniform(0, 1, (6, 9))
    mu = rng.uniform(0.5, 1, 6); mu /= mu.sum()
    nu = rng.uniform(0.5, 1, 9); nu /= nu.sum()
    delta = 1e-6
    nu_cell = nu * (1.0 - delta)
    f, g, P, it, ex = dd.sinkhorn_cell(C, mu, nu_cell, np.zeros(6), 0.2, 1e-12, 100000)
    assert it < 100000
    assert ex == pytest.approx(delta, rel=1e-4)
    np.testing.assert_allclose(P.sum(axis=1), mu * (1.0 - delta), rtol=1e-10)


def test_truncate_keeps_exactly_the_entries_above_the_threshold():
    # Truncate (§6.1, §7.1): after a half-sweep every stored entry of the
    # basic marginals is above the threshold, and the mass reported as
    # truncated is what the Y-marginal lost
    prob = _grid(16, 4, 3, 26)
    eps = 0.004
    rows = dd.product_state(prob)
    alpha = np.zeros(prob.mu.size)
    trunc = 1e-9
    new_rows, info = dd.half_sweep(prob, "A", rows, alpha, eps, dd.Params(err=1e-8, trunc=trunc))
    vals = np.concatenate([v for _, v in new_rows])
    assert vals.min() > trunc
    assert info.truncated_mass > 0
    s = dd.rows_to_dense(new_rows, prob.nu.size).sum(axis=0)
    assert prob.nu.sum() - s.sum() == pytest.approx(info.truncated_mass, rel=1e-6, abs=1e-15)


def test_balance_measures_closed_form():
    # reading R3 by hand: ν_0 = (2, 1) carries 1 too much (target 2), so a
    # third of each entry moves; the deficits 0.25 and 0.75 take a quarter
    # and three quarters of what moved, entry by entry
    parts = [np.array([2.0, 1.0]), np.array([0.5, 0.0]), np.array([0.0, 1.5])]
    out = dd.balance_measures([p.copy() for p in parts], [2.0, 0.75, 2.25])
    moved = np.array([2.0, 1.0]) / 3.0
    np.testing.assert_allclose(out[0], np.array([2.0, 1.0]) - moved, rtol=1e-15)
    np.testing.assert_allclose(out[1], np.array([0.5, 0.0]) + 0.25 * moved, rtol=1e-15)
    np.testing.assert_allclose(out[2], np.array([0.0, 1.5]) + 0.75 * moved, rtol=1e-15)


def test_gather_is_the_sum_on_the_union_of_supports():
    # Algorithm 2: ν_cell = Σ_{i∈J} ν_i, here on hand-made rows
    rows = [(np.array([1, 4, 7]), np.array([0.1, 0.2, 0.3])),
            (np.array([4, 5]), np.array([0.4, 0.5])),
            (np.array([0, 7]), np.array([0.6, 0.7]))]
    cols, nu_cell = dd.gather(rows, [0, 1, 2])
    np.testing.assert_array_equal(cols, [0, 1, 4, 5, 7])
    np.testing.assert_allclose(nu_cell, [0.6, 0.1, 0.6, 0.5, 1.0], rtol=1e-15)
    cols, nu_cell = dd.gather(rows, [1])
    np.testing.assert_array_equal(cols, [4, 5])


def test_refined_marginals_hand_computed():
    # eq. FineBasicMarginals on a case worked out by hand (coarse 4×4 pixels,
    # fine 8×8, b = 2 at both levels, so coarse basic cell (0,0) is the
    # parent of fine basic cells (0,0), (0,1), (1,0), (1,1)):
    #  * fine ν = 1/64 except the children of coarse pixel 1 (fine 2, 3, 10,
    #    11: 1, 2, 3, 2 /64, so ν̂ = 8/64) and of coarse pixel 10 (fine 36,
    #    37, 44, 45: 0.5, 1.5, 1, 1 /64, ν̂ = 4/64);
    #  * fine μ = 1/64 except 3/64 on fine basic cell (0,1), so the parent has
    #    μ̂ = 24/64, fine cell (0,0) 4/64 (share 1/6) and (0,1) 12/64 (1/2);
    #  * coarse row 0 holds 0.06 at coarse pixel 1 and 0.02 at pixel 10.
    # Fine cell (0,0): at the children of pixel 1, ν(y)·(0.06/(8/64))·(1/6) =
    # ν(y)·0.08; at those of pixel 10, ν(y)·(0.02/(4/64))·(1/6) = ν(y)·0.32/6.
    # Fine cell (0,1) gets three times these values; fine cell (1,0) (index 4)
    # the values of (0,0). Coarse row 3 holds 0.05 at coarse pixel 5 (fine
    # children 18, 19, 26, 27 with ν = 1/64, ν̂ = 4/64); its child fine cell
    # (2,2) (index 10) has a quarter of its parent's μ: 0.05/16 each.
    nu_f = np.full((8, 8), 1 / 64)
    nu_f.flat[[2, 3, 10, 11]] = np.array([1, 2, 3, 2]) / 64
    nu_f.flat[[36, 37, 44, 45]] = np.array([0.5, 1.5, 1, 1]) / 64
    mu_f = np.full((8, 8), 1 / 64)
    mu_f[0:2, 2:4] = 3 / 64
    coarse = dd.GridProblem(dd.pyramid(mu_f, 2)[0], dd.pyramid(nu_f, 2)[0], 2, 1 / 4)
    fine = dd.GridProblem(mu_f, nu_f, 2, 1 / 8)
    rows_c = [(np.array([1, 10]), np.array([0.06, 0.02])), (np.array([0]), np.array([0.01])),
              (np.array([15]), np.array([0.01])), (np.array([5]), np.array([0.05]))]
    rows_f = dd.refine_basic_marginals(coarse, fine, rows_c)
    y0 = [2, 3, 10, 11, 36, 37, 44, 45]
    v0 = [0.00125, 0.0025, 0.00375, 0.0025, 0.0004166666666666667, 0.00125, 0.0008333333333333334,
          0.0008333333333333334]
    v1 = [0.00375, 0.0075, 0.01125, 0.0075, 0.00125, 0.00375, 0.0025, 0.0025]
    for i, v in ((0, v0), (1, v1), (4, v0)):
        np.testing.assert_array_equal(rows_f[i][0], y0)
        np.testing.assert_allclose(rows_f[i][1], v, rtol=1e-13)
    np.testing.assert_array_equal(rows_f[10][0], [18, 19, 26, 27])
    np.testing.assert_allclose(rows_f[10][1], [0.003125] * 4, rtol=1e-13)


def test_fill_massless_affine_reproduces_an_affine_dual():
    # pixels without mass take the affine fit of their A cell's dual: on an
    # affine α (a different plane per A cell) they get exactly its values,
    # and pixels with mass keep theirs
    n, b = 16, 4
    mu = syn.gaussian_mixture(n, 2, 12)
    dead = [(0, 0), (7, 7), (3, 4), (8, 15), (12, 9)]
    for r, c in dead:
        mu[r, c] = 0.0
    prob = dd.GridProblem(mu, syn.gaussian_mixture(n, 2, 13), b, 1 / n)
    i, j = np.divmod(np.arange(n * n), n)
    cell = (i // (2 * b)) * (n // (2 * b)) + j // (2 * b)
    rng = np.random.default_rng(5)
    a, sr, sc = rng.normal(size=(3, cell.max() + 1))
    alpha = a[cell] + sr[cell] * i + sc[cell] * j
    scrambled = alpha.copy()
    for r, c in dead:
        scrambled[r * n + c] = 1e3 * rng.normal()
    out = dd.fill_massless_affine(prob, scrambled)
    np.testing.assert_allclose(out, alpha, rtol=0, atol=1e-11)
    live = prob.mu > 0
    np.testing.assert_array_equal(out[live], scrambled[live])


def _cell_optimum(prob, rows, J, e):
    """The cell problem's entropic optimum at ε = e, solved from zero duals
    to a tight tolerance (independent of any warm start)."""
    cols, nu_cell = dd.gather(rows, J)
    X = prob.cell_points(J)
    live = prob.mu[X] > 0
    C = prob.cost(X[live], cols)
    _, _, P, _, _ = dd.sinkhorn_cell(C, prob.mu[X][live], nu_cell, np.zeros(int(live.sum())), e, 1e-12, 200000)
    return P


def test_safeguard_keeps_the_cell_optimum_of_a_larger_eps():
    # §7.3 safeguard: a cold start at a small ε with 60 iterations per solve;
    # every cell fails at ε and is kept at 4ε or 16ε. The kept plan is the
    # cell problem's optimum at that ε (an independent tight solve), and the
    # state stays feasible (Σ_i ν_i = ν, ‖ν_i‖ = ‖μ_i‖)
    n, eps = 16, 0.002
    mu = syn.gaussian_mixture(n, 3, 60)
    nu = syn.gaussian_mixture(n, 3, 61)
    prob = dd.GridProblem(mu / mu.sum(), nu / nu.sum(), 4, 1.0 / n)
    rows = dd.product_state(prob)
    plans = {}
    new_rows, info = dd.half_sweep(prob, "A", rows, np.zeros(n * n), eps,
                                   dd.Params(err=1e-6, max_iter=60, safeguard=True), plans=plans)
    assert info.rescued == 4 and info.escalated == 4 and all(info.converged)
    assert sorted({round(e / eps) for e in info.eps_used}) == [4, 16]
    for jn, J in enumerate(prob.parts["A"]):
        X, cols, P = plans[jn]
        live = prob.mu[X] > 0
        want = _cell_optimum(prob, rows, J, info.eps_used[jn])
        assert np.abs(P[live] - want).sum() <= 1e-4 * want.sum()
    assert dd.y_marginal_error(prob, new_rows) <= info.truncated_mass + 1e-14
    for i, (c, v) in enumerate(new_rows):
        if i in {k for J in prob.parts["A"] for k in J}:
            assert abs(v.sum() - prob.basic_mass[i]) <= 1e-13
    # without the safeguard the same solves stop at max_iter far from the tolerance
    _, info0 = dd.half_sweep(prob, "A", rows, np.zeros(n * n), eps, dd.Params(err=1e-6, max_iter=60))
    assert not any(info0.converged) and info0.rescued == 0


def test_safeguard_rescues_a_forced_failure_at_eps():
    # the first solve of every cell cut off after one iteration (from duals
    # converged at 2ε, far from the ε optimum): the safeguard solves at 4ε,
    # then at ε, and keeps ε; the result is the plain half-sweep's at ε
    n, eps = 16, 0.004
    mu = syn.gaussian_mixture(n, 3, 62)
    nu = syn.gaussian_mixture(n, 3, 63)
    prob = dd.GridProblem(mu / mu.sum(), nu / nu.sum(), 4, 1.0 / n)
    rows = dd.product_state(prob)
    alpha = np.zeros(n * n)
    p = dd.Params(err=1e-9, max_iter=20000)
    for _ in range(6):
        rows, _ = dd.half_sweep(prob, "A", rows, alpha, 2 * eps, p)
        rows, _ = dd.half_sweep(prob, "B", rows, alpha, 2 * eps, p)
    a_plain, a_safe = alpha.copy(), alpha.copy()
    want, _ = dd.half_sweep(prob, "A", rows, a_plain, eps, dd.Params(err=1e-9, max_iter=20000))
    got, info = dd.half_sweep(prob, "A", rows, a_safe, eps,
                              dd.Params(err=1e-9, max_iter=20000, safeguard=True, main_max_iter=1))
    assert info.rescued == 4 and info.escalated == 0 and all(info.converged)
    assert all(e == eps for e in info.eps_used)
    D1, D2 = dd.rows_to_dense(got, n * n), dd.rows_to_dense(want, n * n)
    assert np.abs(D1 - D2).sum() <= 1e-7
