"""The hybrid dual refinement (dd_options.dual_refine = 1: A cells from the
cell-wise refinement, B cells from the glued coarse dual interpolated
linearly, §6.3–6.4) against the oracle's run with the same refinement. This
file is collected last so that a failure here does not hide other tests.
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
