"""dd_objective against the oracle: the primal score KL(π|K) − ‖K‖ summed
cell by cell (§6.3) and the primal-dual gaps of the cell problems
(Prop. 2.5, eq. EntropicOTDualObjective). This file is collected after the
other GPU parity tests so that a failure here does not hide them.
"""
import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


@pytest.fixture(scope="module")
def ref32():
    mu = syn.gaussian_mixture(32, 3, 50)
    nu = syn.gaussian_mixture(32, 3, 51)
    sched = [(0.004, 4, 0)]
    return mu, nu, sched, odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))


def test_objective_of_a_given_state_matches_oracle(lib):
    # the primal score KL(π|K) − ‖K‖ and the cell problems' primal-dual gaps
    # (§6.3, Prop. 2.5) of the coupling that a feasible synthetic state with
    # random duals gives, both partitions, against the oracle on the same state
    n, b, eps = 32, 4, 0.004
    mu = syn.gaussian_mixture(n, 3, 80)
    nu, rp, col, val = syn.feasible_state(mu, b, seed=9, radius_px=4)
    rng = np.random.default_rng(10)
    alphas = [eps * rng.normal(0.0, 0.5, n * n), eps * rng.normal(0.0, 0.5, n * n)]
    g = lib.DD(mu, nu, b, 1, [(eps, 1, 0)])
    g.set_state(rp, col, val, alphas[0], alphas[1])
    got = [g.objective(p, eps) for p in (0, 1)]
    g.close()
    prob = odd.GridProblem(mu / mu.sum(), nu / nu.sum(), b, 1.0 / n)
    rows = odd.rows_from_csr(rp, col, val / nu.sum())
    for p, part in enumerate("AB"):
        primal, gap = odd.cell_objectives(prob, part, rows, alphas[p], eps)
        pr, gs, ga = got[p]
        assert abs(gap).sum() > 1e-3                  # far from the cell optima
        assert pr == pytest.approx(primal.sum(), rel=1e-5), (p, pr, primal.sum())
        assert gs == pytest.approx(gap.sum(), rel=1e-4, abs=1e-5 * abs(gap).sum())
        assert ga == pytest.approx(abs(gap).sum(), rel=1e-4)


def test_objective_after_the_schedule_matches_oracle(lib, ref32):
    # converged state of the 32² run: primal score against the oracle's, and
    # the cell gaps small against it (Table 1 reports relative primal-dual
    # gaps near 1e-4)
    mu, nu, sched, ref = ref32
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-7)
    g.run_schedule()
    pr, gs, ga = g.objective()
    with pytest.raises(lib.DDError):
        g.objective(2, 0.004)
    g.close()
    primal, gap = odd.cell_objectives(ref.prob, ref.last_part, ref.rows, ref.alpha[ref.last_part], ref.eps)
    assert pr == pytest.approx(primal.sum(), rel=1e-5)
    assert ga < 1e-5 * abs(primal.sum())
    assert abs(gap).sum() < 1e-7 * abs(primal.sum())
