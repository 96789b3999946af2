"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (from the targets of the method's GPU form): basic marginals and
pixel-level plan ≤ 1e-5 relative L1, transport cost ≤ 1e-6 relative, marginal
errors ≤ 1e-6 L1. The GPU computes potentials in FP32; the oracle in FP64 with
a tighter Sinkhorn tolerance.
"""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-5
COST_TOL = 1e-6
MARG_TOL = 1e-6


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def _rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def _dense_rows(rp, col, val, ny):
    return odd.rows_to_dense(odd.rows_from_csr(rp, col, val), ny)


def _dense_plan(rp, col, val, nx, ny):
    P = np.zeros((nx, ny))
    for x in range(nx):
        P[x, col[rp[x]:rp[x + 1]]] = val[rp[x]:rp[x + 1]]
    return P


def _compare_run(lib, mu, nu, b, levels, sched, gpu_err=1e-6, oracle_err=1e-10, check_plan=True,
                 threads=0):
    n = mu.shape[0]
    g = lib.DD(mu, nu, b, levels, sched, err_tol=gpu_err, threads_per_cell=threads)
    st = g.run_schedule()
    rp, col, val = g.basic_marginals()
    cost, ex, ey = g.cost()
    level, nl, _, eps, _ = g.info()
    plan = g.plan(0.0) if check_plan else None
    g.close()
    ref = odd.run_schedule(mu, nu, b, levels, sched, odd.Params(err=oracle_err))
    assert nl == ref.prob.n
    ny = nl * nl
    got = _dense_rows(rp, col, val, ny)
    exp = odd.rows_to_dense(ref.rows, ny)
    info = ref.history[-1][3]
    out = dict(rows=_rel_l1(got, exp), cost=abs(cost - info.cost) / info.cost, err_x=ex, err_y=ey,
               ref_err_y=odd.y_marginal_error(ref.prob, ref.rows), stats=st)
    if check_plan:
        P = _dense_plan(*plan, ny, ny)
        Pref = odd.partition_plan(ref.prob, ref.last_part, ref.rows, ref.alpha[ref.last_part], ref.eps)
        out["plan"] = _rel_l1(P, Pref)
    return out


def test_single_cell_is_sinkhorn(lib):
    # n = 2b: partition A is one cell, so one A half-sweep is a full Sinkhorn solve
    n, b, eps = 8, 4, 0.02
    mu = syn.gaussian_mixture(n, 2, 0)
    nu = syn.gaussian_mixture(n, 2, 1)
    g = lib.DD(mu, nu, b, 1, [(eps, 1, 0)], err_tol=1e-6)
    g.half_sweep(0, eps)
    P = _dense_plan(*g.plan(0.0), n * n, n * n)
    g.close()
    prob = odd.GridProblem(mu, nu, b, 1.0 / n)
    alpha = np.zeros(n * n)
    rows, _ = odd.half_sweep(prob, "A", odd.product_state(prob), alpha, eps, odd.Params(err=1e-12))
    Pref = odd.partition_plan(prob, "A", rows, alpha, eps)
    assert _rel_l1(P, Pref) < PLAN_TOL


def test_config1_full_schedule(lib):
    # two 32×32 images of 3 blobs, 4×4 cells, ε halving 1.0 → 2h², 20 sweeps each
    mu, nu = syn.image_pair("gm32_b4", 0)
    sched = syn.halving_schedule(1.0, 2.0 / 32**2, 20)
    r = _compare_run(lib, mu, nu, 4, 1, sched, gpu_err=1e-6, oracle_err=1e-8)
    assert r["rows"] < PLAN_TOL, r
    assert r["plan"] < PLAN_TOL, r
    assert r["cost"] < COST_TOL, r
    assert r["err_x"] < MARG_TOL and r["err_y"] < MARG_TOL, r


def test_ragged_grid_fixed_eps(lib):
    # 24×24 with 4×4 cells: 6×6 basic cells, B has corner, edge and full cells
    mu = syn.gaussian_mixture(24, 3, 20)
    nu = syn.gaussian_mixture(24, 3, 21)
    r = _compare_run(lib, mu, nu, 4, 1, [(0.004, 12, 0)], gpu_err=1e-6)
    assert r["rows"] < PLAN_TOL and r["plan"] < PLAN_TOL and r["cost"] < COST_TOL, r


def test_two_levels_refinement(lib):
    # 16² → 32² with the paper's per-level schedule, then 6 sweeps at 2h²
    mu = syn.gaussian_mixture(32, 4, 30)
    nu = syn.gaussian_mixture(32, 4, 31)
    sched = syn.paper_schedule(32, 2, 6)
    r = _compare_run(lib, mu, nu, 4, 2, sched, gpu_err=1e-6, oracle_err=1e-9)
    assert r["rows"] < PLAN_TOL and r["cost"] < COST_TOL, r
    assert r["err_y"] < MARG_TOL, r


@pytest.mark.parametrize("b,n,eps,sweeps", [(8, 32, 0.004, 2), (2, 16, 0.01, 4)])
def test_cell_sizes(lib, b, n, eps, sweeps):
    mu = syn.gaussian_mixture(n, 3, 40 + b)
    nu = syn.gaussian_mixture(n, 3, 41 + b)
    r = _compare_run(lib, mu, nu, b, 1, [(eps, sweeps, 0)], gpu_err=1e-6, oracle_err=1e-9)
    assert r["rows"] < PLAN_TOL and r["cost"] < COST_TOL, r


@pytest.fixture(scope="module")
def ref32():
    mu = syn.gaussian_mixture(32, 3, 50)
    nu = syn.gaussian_mixture(32, 3, 51)
    sched = [(0.004, 4, 0)]
    return mu, nu, sched, odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))


@pytest.mark.parametrize("threads,clusters", [(64, 0), (128, 0), (256, 0), (128, 4), (128, 32)])
def test_threads_and_clusters(lib, ref32, threads, clusters):
    # per-CTA cell solves with 64/128/256 threads, and cluster solves of the
    # 4 or all largest cells (8 CTAs sharing one cell)
    mu, nu, sched, ref = ref32
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-7, threads_per_cell=threads, max_cluster_cells=clusters)
    g.run_schedule()
    rp, col, val = g.basic_marginals()
    cost, _, _ = g.cost(with_y=False)
    g.close()
    got = _dense_rows(rp, col, val, 32 * 32)
    assert _rel_l1(got, odd.rows_to_dense(ref.rows, 32 * 32)) < PLAN_TOL
    assert abs(cost - ref.history[-1][3].cost) / ref.history[-1][3].cost < COST_TOL


def test_duals_match_up_to_cell_constants(lib, ref32):
    mu, nu, sched, ref = ref32
    eps = sched[0][0]
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-7)
    g.run_schedule()
    aA, aB = g.duals(0), g.duals(1)
    g.close()
    for part, a in (("A", aA), ("B", aB)):
        for J in ref.prob.parts[part]:
            X = ref.prob.cell_points(J)
            d = a[X] - ref.alpha[part][X]
            assert np.ptp(d) / eps < 1e-3


def test_sampled_cells_full_size(lib):
    # 1024² images, 4×4 cells: a feasible synthetic state, one A half-sweep at
    # ε = 2h², compared on a sample of cells that the oracle solves one by one
    n, b = 1024, 4
    eps = 2.0 / n**2
    mu, _ = syn.image_pair("gm1024_b4", 0)
    nu, rp, col, val = syn.feasible_state(mu, b, seed=7)
    g = lib.DD(mu, nu, b, 1, [(eps, 1, 0)], err_tol=1e-6)
    g.set_state(rp, col, val)
    g.half_sweep(0, eps)
    grp, gcol, gval = g.basic_marginals()
    g.close()
    prob = odd.GridProblem(mu / mu.sum(), nu / nu.sum(), b, 1.0 / n)
    rows = odd.rows_from_csr(rp, col, val / nu.sum())
    rng = np.random.default_rng(3)
    cells = sorted(rng.choice(len(prob.parts["A"]), 48, replace=False).tolist())
    cells += [0, len(prob.parts["A"]) - 1]
    new_rows, _ = odd.half_sweep(prob, "A", rows, np.zeros(n * n), eps, odd.Params(err=1e-10), cells=cells)
    num = den = 0.0
    for jn in cells:
        for i in prob.parts["A"][jn]:
            c_ref, v_ref = new_rows[i]
            c_gpu = gcol[grp[i]:grp[i + 1]]
            v_gpu = gval[grp[i]:grp[i + 1]]
            u = np.union1d(c_ref, c_gpu)
            a = np.zeros(u.size); a[np.searchsorted(u, c_gpu)] = v_gpu
            e = np.zeros(u.size); e[np.searchsorted(u, c_ref)] = v_ref
            num += np.abs(a - e).sum()
            den += e.sum()
    assert num / den < PLAN_TOL, num / den


def test_sampled_cells_full_size_with_cluster_cells(lib):
    # 1024², 4×4 cells: a feasible synthetic state in which three basic cells
    # send their mass to wide bumps, so that their composite cells get
    # supports large enough for the 8-CTA cluster solver; one A half-sweep at
    # ε = 2h², compared on every cluster-solved cell and a random sample of
    # the others: basic marginals (relative L1) and each cell's transport cost
    n, b = 1024, 4
    eps = 2.0 / n**2
    mu, _ = syn.image_pair("gm1024_b4", 0)
    _, rp0, col0, val0 = syn.feasible_state(mu, b, seed=7, radius_px=3)
    _, rpw, colw, valw = syn.feasible_state(mu, b, seed=7, radius_px=26, blur_px=8.0)
    nb = n // b
    wide = {100 * nb + 100, 180 * nb + 62, 40 * nb + 200}
    rows = []
    for i in range(nb * nb):
        rp, col, val = (rpw, colw, valw) if i in wide else (rp0, col0, val0)
        rows.append((col[rp[i]:rp[i + 1]].astype(np.int64), val[rp[i]:rp[i + 1]]))
    nu = np.zeros(n * n)
    for c, v in rows:
        nu[c] += v
    rp = np.zeros(nb * nb + 1, dtype=np.int64)
    rp[1:] = np.cumsum([c.size for c, _ in rows])
    col = np.concatenate([c for c, _ in rows]).astype(np.int32)
    val = np.concatenate([v for _, v in rows])
    g = lib.DD(mu, nu.reshape(n, n), b, 1, [(eps, 1, 0)], err_tol=1e-6)
    g.set_state(rp, col, val)
    g.half_sweep(0, eps)
    grp, gcol, gval = g.basic_marginals()
    cs = g.cell_stats()
    g.close()
    clusters = np.flatnonzero(cs["cluster"]).tolist()
    wide_cells = sorted({(i // nb // 2) * (nb // 2) + (i % nb) // 2 for i in wide})
    assert set(wide_cells) <= set(clusters), (wide_cells, clusters[:10])
    prob = odd.GridProblem(mu / mu.sum(), nu.reshape(n, n) / nu.sum(), b, 1.0 / n)
    orows = odd.rows_from_csr(rp, col, val / nu.sum())
    rng = np.random.default_rng(5)
    cells = sorted(set(rng.choice(len(prob.parts["A"]), 24, replace=False).tolist()) | set(clusters[:8]))
    plans = {}
    new_rows, _ = odd.half_sweep(prob, "A", orows, np.zeros(n * n), eps, odd.Params(err=1e-10, max_iter=100000),
                                 cells=cells, plans=plans)
    num = den = 0.0
    got_cost = ref_cost = 0.0
    for jn in cells:
        for i in prob.parts["A"][jn]:
            c_ref, v_ref = new_rows[i]
            c_gpu, v_gpu = gcol[grp[i]:grp[i + 1]], gval[grp[i]:grp[i + 1]]
            u = np.union1d(c_ref, c_gpu)
            a = np.zeros(u.size); a[np.searchsorted(u, c_gpu)] = v_gpu
            e = np.zeros(u.size); e[np.searchsorted(u, c_ref)] = v_ref
            num += np.abs(a - e).sum()
            den += e.sum()
        X, ycols, P = plans[jn]
        cj = float((prob.cost(X, ycols) * P).sum())
        # one cell solved to Err = 1e-6 moves its cost by up to about that much
        assert abs(cs["cost"][jn] - cj) / cj < 10 * COST_TOL, (jn, cs["cost"][jn], cj)
        got_cost += cs["cost"][jn]
        ref_cost += cj
    assert num / den < PLAN_TOL, num / den
    assert abs(got_cost - ref_cost) / ref_cost < COST_TOL


def test_set_state_rejects_unsorted(lib):
    n, b = 16, 4
    mu = syn.gaussian_mixture(n, 2, 70)
    nu, rp, col, val = syn.feasible_state(mu, b, seed=1, radius_px=2)
    g = lib.DD(mu, nu, b, 1, [(0.01, 1, 0)])
    bad = col.copy()
    bad[rp[0]], bad[rp[0] + 1] = bad[rp[0] + 1], bad[rp[0]]
    with pytest.raises(lib.DDError) as e:
        g.set_state(rp, bad, val)
    assert e.value.status == lib.DD_ERR_ARG
    g.set_state(rp, col, val)           # the context is still usable
    g.half_sweep(1, 0.01)
    g.close()


@pytest.fixture(scope="module")
def ref_spread():
    # a narrow blob spread over a wide one at ε = h²: cells whose X-iteration
    # contracts slowly (the oracle needs 130–550 iterations per cell)
    mu = syn.gaussian_mixture(16, 1, 60, sigma_range=(0.05, 0.06))
    nu = syn.gaussian_mixture(16, 2, 61, sigma_range=(0.3, 0.35))
    sched = [(1.0 / 256, 4, 0)]
    return mu, nu, sched, odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))


@pytest.mark.parametrize("newton", [1, 0])
def test_newton_x_iteration_matches_oracle(lib, ref_spread, newton):
    # with Newton X-iterations on, such cells take Newton steps; on or off, the
    # result is the oracle's fixed point
    mu, nu, sched, ref = ref_spread
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-7, x_newton=newton)
    g.run_schedule()
    prof = g.profile()
    rp, col, val = g.basic_marginals()
    cost, _, _ = g.cost(with_y=False)
    g.close()
    assert (prof.newton_steps > 0) == bool(newton), prof.newton_steps
    got = _dense_rows(rp, col, val, 16 * 16)
    assert _rel_l1(got, odd.rows_to_dense(ref.rows, 16 * 16)) < PLAN_TOL
    assert abs(cost - ref.history[-1][3].cost) / ref.history[-1][3].cost < COST_TOL


def test_graph_mode_matches_oracle_and_per_kernel_mode(lib, ref32):
    # mode 1: persistent per-CTA solves and sweeps 2..4 replayed from a captured
    # graph; the cells are solved by the same arithmetic, so the state equals
    # the per-kernel mode's bit for bit
    mu, nu, sched, ref = ref32
    out = {}
    for mode in (0, 1):
        g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-7, mode=mode)
        g.run_schedule()
        out[mode] = (g.basic_marginals(), g.cost(with_y=False)[0], g.profile().half_sweeps)
        g.close()
    (rp0, c0, v0), cost0, hs0 = out[0]
    (rp1, c1, v1), cost1, hs1 = out[1]
    assert hs0 == hs1 == 8
    assert np.array_equal(rp0, rp1) and np.array_equal(c0, c1) and np.array_equal(v0, v1)
    assert cost0 == cost1
    got = _dense_rows(rp1, c1, v1, 32 * 32)
    assert _rel_l1(got, odd.rows_to_dense(ref.rows, 32 * 32)) < PLAN_TOL


def test_autotune_picks_a_candidate_and_keeps_the_state_feasible(lib):
    # 9 tuning sweeps are real sweeps: the state stays feasible and converges
    mu = syn.gaussian_mixture(32, 3, 70)
    nu = syn.gaussian_mixture(32, 3, 71)
    g = lib.DD(mu, nu, 4, 1, [(0.004, 2, 0)], err_tol=1e-7, mode=1)
    g.run_schedule()
    t, cl = g.autotune(rounds=1)
    assert t in (64, 128, 256) and cl in (0, 64, 256)
    assert g.profile().half_sweeps == 2 * (2 + 9)
    cost, ex, ey = g.cost()
    g.close()
    assert ey < 1e-9 and ex < 1e-5 and cost > 0   # ey: mass dropped by Truncate


def test_zero_mass_pixels(lib):
    # pixels without mass (inside basic cells that have mass) in μ and in ν:
    # their potentials are −∞ in the oracle; the plan must still match
    n, b, eps = 16, 4, 0.01
    mu = syn.gaussian_mixture(n, 2, 90)
    nu = syn.gaussian_mixture(n, 2, 91)
    mu[3, 5] = mu[9, 9] = mu[12, 0] = 0.0
    nu[0, 0] = nu[7, 8] = nu[15, 15] = 0.0
    mu /= mu.sum()
    nu /= nu.sum()
    sched = [(eps, 3, 0)]
    with np.errstate(divide="ignore"):
        ref = odd.run_schedule(mu, nu, b, 1, sched, odd.Params(err=1e-10))
    g = lib.DD(mu, nu, b, 1, sched, err_tol=1e-7)
    g.run_schedule()
    rp, col, val = g.basic_marginals()
    cost, ex, ey = g.cost()
    g.close()
    got = _dense_rows(rp, col, val, n * n)
    want = odd.rows_to_dense(ref.rows, n * n)
    assert np.all(got[:, [0, 7 * n + 8, n * n - 1]] == 0.0)
    assert _rel_l1(got, want) < PLAN_TOL
    assert abs(cost - ref.history[-1][3].cost) / ref.history[-1][3].cost < COST_TOL
