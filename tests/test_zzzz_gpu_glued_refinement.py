"""Dual gluing on GPU runs (§6.3–6.4): the hybrid dual refinement
(dd_options.dual_refine = 1: A cells from the cell-wise refinement, B cells
from the glued coarse dual interpolated linearly) against the oracle's run
with the same refinement, and eq. RelPDGap of a GPU state against the
oracle's. This file is collected last so that a failure here does not hide
other tests.
"""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-5
COST_TOL = 1e-6


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def test_hybrid_refinement_matches_oracle(lib):
    # 16² → 32² with the paper's per-level schedule, then 6 sweeps at 2h²
    mu = syn.gaussian_mixture(32, 4, 30)
    nu = syn.gaussian_mixture(32, 4, 31)
    sched = syn.paper_schedule(32, 2, 6)
    g = lib.DD(mu, nu, 4, 2, sched, err_tol=1e-6, dual_refine=1)
    g.run_schedule()
    rp, col, val = g.basic_marginals()
    cost, _, _ = g.cost(with_y=False)
    g.close()
    ref = odd.run_schedule(mu, nu, 4, 2, sched, odd.Params(err=1e-9), dual_refinement="hybrid")
    got = odd.rows_to_dense(odd.rows_from_csr(rp, col, val), 32 * 32)
    want = odd.rows_to_dense(ref.rows, 32 * 32)
    assert np.abs(got - want).sum() / want.sum() < PLAN_TOL
    ref_cost = ref.history[-1][3].cost
    assert abs(cost - ref_cost) / ref_cost < COST_TOL


def test_relative_pd_gap_of_a_gpu_run(lib):
    # eq. RelPDGap after the multi-scale schedule (16² → 32², 6 final sweeps):
    # duals and coupling from the GPU, gluing and gap on the host, against the
    # oracle's dense evaluation of its own run of the same schedule (1.5e-7
    # there; a few sweeps at one ε from the product coupling leave a gap of
    # several percent, so the schedule matters)
    mu = syn.gaussian_mixture(32, 4, 30)
    nu = syn.gaussian_mixture(32, 4, 31)
    sched = syn.paper_schedule(32, 2, 6)
    g = lib.DD(mu, nu, 4, 2, sched, err_tol=1e-6)
    g.run_schedule()
    rel, gap, primal = g.relative_pd_gap(mu, nu)
    g.close()
    ref = odd.run_schedule(mu, nu, 4, 2, sched, odd.Params(err=1e-9))
    a_hat, _ = odd.glue_duals(ref.prob, ref.alpha["A"], ref.alpha["B"], ref.eps)
    b_hat = odd.best_y_dual(ref.prob, a_hat, ref.eps)
    P = odd.partition_plan(ref.prob, ref.last_part, ref.rows, ref.alpha[ref.last_part], ref.eps)
    rel_w, _, primal_w = odd.relative_pd_gap(ref.prob, P, a_hat, b_hat, ref.eps)
    assert primal == pytest.approx(primal_w, rel=1e-5)
    assert abs(rel) < 1e-4 and abs(rel - rel_w) < 1e-5


def test_hybrid_refinement_duals_with_massless_corners(lib):
    # pixels without mass at corners of coarse A and B cells: the glued coarse
    # dual is continued there by the affine fit of its A cell before the §6.4
    # interpolation, so the B duals of the fine level match the oracle's on
    # every pixel with mass (up to one constant per cell), and the run still
    # converges to the oracle's state
    n, b = 32, 4
    mu = syn.gaussian_mixture(n, 4, 32)
    nu = syn.gaussian_mixture(n, 4, 33)
    for (r, c) in ((0, 0), (7, 7), (4, 4), (8, 4)):      # coarse pixels (16² level)
        mu[2 * r:2 * r + 2, 2 * c:2 * c + 2] = 0.0
    mu /= mu.sum()
    sched = syn.paper_schedule(n, 2, 6)
    coarse = [s for s in sched if s[2] == 0]
    n0 = sum(s[1] for s in coarse)
    g = lib.DD(mu, nu, b, 2, sched, err_tol=1e-7, dual_refine=1)
    g.sweep(n0)
    g.refine()
    aB = g.duals(1)
    with np.errstate(divide="ignore"):
        ref_c = odd.run_schedule(mu, nu, b, 2, coarse, odd.Params(err=1e-10))
    fine = odd.GridProblem(mu, nu, b, 1.0 / n)
    a_hat, _ = odd.glue_duals(ref_c.prob, ref_c.alpha["A"], ref_c.alpha["B"], ref_c.eps)
    a_ref = odd.refine_duals_glued(ref_c.prob, fine, odd.fill_massless_affine(ref_c.prob, a_hat))
    eps_f = sched[len(coarse)][0]
    worst = 0.0
    for J in fine.parts["B"]:
        X = fine.cell_points(J)
        X = X[fine.mu[X] > 0]
        worst = max(worst, np.ptp(aB[X] - a_ref[X]) / eps_f)
    assert worst < 1e-3, worst
    g.sweep(sum(s[1] for s in sched) - n0)
    rp, col, val = g.basic_marginals()
    cost, _, _ = g.cost(with_y=False)
    g.close()
    with np.errstate(divide="ignore"):
        ref = odd.run_schedule(mu, nu, b, 2, sched, odd.Params(err=1e-9), dual_refinement="hybrid")
    got = odd.rows_to_dense(odd.rows_from_csr(rp, col, val), n * n)
    want = odd.rows_to_dense(ref.rows, n * n)
    assert np.abs(got - want).sum() / want.sum() < PLAN_TOL
    ref_cost = ref.history[-1][3].cost
    assert abs(cost - ref_cost) / ref_cost < COST_TOL


@pytest.mark.parametrize("n,levels,blank", [(80, 1, False), (256, 3, True)])
def test_device_gluing_matches_host_and_oracle(lib, n, levels, blank):
    # the A-cell grid split over the 8 CTAs of the gluing's CG cluster: 10
    # rows (five CTAs with two rows, three with none) and 32 rows (four
    # each); at 256² some pixels without mass, which get α̂ = 0
    b = 4
    mu = syn.gaussian_mixture(n, 4, 80)
    nu = syn.gaussian_mixture(n, 4, 81)
    if blank:
        for (r, c) in ((0, 0), (17, 30), (100, 101), (255, 128)):
            mu[r, c] = 0.0
        mu /= mu.sum()
    sched = ([(0.02, 2, 0), (0.01, 2, 0), (0.005, 3, 0)] if levels == 1
             else syn.paper_schedule(n, levels, 1))
    g = lib.DD(mu, nu, b, levels, sched, err_tol=1e-6)
    g.run_schedule()
    _, nl, _, eps, _ = g.info()
    assert nl == n
    aA, aB = g.duals(0), g.duals(1)
    a_gpu, V_gpu, it, rr = g.glue_duals()
    g.close()
    m = (mu / mu.sum()).reshape(-1)
    a_host, V_host = lib.dd_glue_duals_host(m.reshape(n, n), aA, aB, b, eps)
    prob = odd.GridProblem(mu / mu.sum(), nu / nu.sum(), b, 1.0 / n)
    a_or, V_or = odd.glue_duals(prob, aA, aB, eps)
    assert it > 0 and rr <= 1e-13
    assert np.all(a_gpu[m == 0] == 0.0)
    for V_ref, a_ref in ((V_host, a_host), (V_or, a_or)):
        scale = 1.0 + np.abs(V_ref).max()
        assert np.abs(V_gpu - V_ref).max() <= 1e-9 * scale
        assert np.abs(a_gpu - np.ravel(a_ref)).max() / eps <= 1e-9 * scale


def test_device_relative_pd_gap_matches_host(lib):
    # the same state evaluated on the GPU and on the host (downloaded duals,
    # host gluing, dd_get_plan's coupling without truncation): the entries
    # are the same FP32 exponentials, the logs differ by their FP32 rounding
    n = 64
    mu = syn.gaussian_mixture(n, 5, 82)
    nu = syn.gaussian_mixture(n, 5, 83)
    sched = syn.paper_schedule(n, 2, 4)
    g = lib.DD(mu, nu, 4, 2, sched, err_tol=1e-6)
    g.run_schedule()
    rel_d, gap_d, pr_d = g.relative_pd_gap()
    rel_h, gap_h, pr_h = g.relative_pd_gap(mu / mu.sum(), nu / nu.sum(), device=False)
    # a second call gives the same primal and, up to the order of the atomic
    # additions, the same gap
    rel_d2, _, pr_d2 = g.relative_pd_gap()
    g.close()
    assert pr_d == pytest.approx(pr_h, rel=1e-5)
    assert abs(rel_d - rel_h) < 2e-6, (rel_d, rel_h)
    assert pr_d2 == pr_d and abs(rel_d2 - rel_d) < 1e-12
    assert rel_d > 0.0


def test_hybrid_refinement_on_device_matches_host_gluing(lib):
    # 64² → 128² → 256²: at the last refinement the 128² level has 16 rows of
    # A cells (two per CTA of the CG cluster); the B duals of the 256² level
    # from the device path and from the host path (debug_flags bit 5) agree,
    # and so do the states after the rest of the schedule
    n = 256
    mu = syn.gaussian_mixture(n, 5, 84)
    nu = syn.gaussian_mixture(n, 5, 85)
    sched = syn.paper_schedule(n, 3, 2)
    n0 = sum(s[1] for s in sched if s[2] < 2)
    out = {}
    for flags in (0, 32):
        g = lib.DD(mu, nu, 4, 3, sched, err_tol=1e-6, dual_refine=1, debug_flags=flags)
        g.sweep(n0)
        g.refine()
        eps_f = sched[[s[2] for s in sched].index(2)][0]
        aB = g.duals(1)
        g.sweep(sum(s[1] for s in sched) - n0)
        cost, ex, ey = g.cost()
        out[flags] = (aB, cost, ex, ey)
        g.close()
    live = (mu > 0).reshape(-1)
    d = np.abs(out[0][0] - out[32][0])[live].max() / eps_f
    assert d < 1e-5, d
    assert abs(out[0][1] - out[32][1]) / out[32][1] < 1e-7
    assert out[0][2] < 1e-5 and out[0][3] < 1e-9
