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
