"""Checkpoint/resume, the local safeguard of §7.3, the non-convergence status
and host-side fault injection (dd_options.debug_flags bits 2–4) on the GPU.

No test here faults or hangs the GPU: the injected failures are made on the
host (a buffer sized too small on purpose, a solve cut off after one
iteration, an allocation reported as failed before it is made).
"""
import warnings

import numpy as np
import pytest

from oracle import dd as odd
from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

PLAN_TOL = 1e-5
COST_TOL = 1e-6
# ε halved from 0.05 to 0.00625, two sweeps each, and Err = 1e-6: every cell
# solve starts warm and its tolerance lies above the FP32 floor of the
# X-marginal error, so none needs more than max_iter iterations (a cold start
# at a small ε, or Err = 1e-7, can leave a few cells at max_iter)
WARM_SCHEDULE = [(0.05, 2, 0), (0.025, 2, 0), (0.0125, 2, 0), (0.00625, 2, 0)]


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2001_10986_gb300 import build
    build.build()
    from paper_2001_10986_gb300 import dd
    return dd


def _state(g):
    rp, col, val = g.basic_marginals()
    return rp, col, val, g.duals(0), g.duals(1), g.cost(with_y=False)[0]


def _assert_same_state(s1, s2):
    for a, b in zip(s1[:5], s2[:5]):
        assert np.array_equal(a, b)
    assert s1[5] == s2[5]


@pytest.mark.parametrize("mode", [0, 1])
def test_checkpoint_resume_is_bit_identical(lib, tmp_path, mode):
    # 16² → 32²: save in the middle of the coarse level's schedule and at the
    # fine level; the resumed context reaches the uninterrupted run's state
    mu = syn.gaussian_mixture(32, 4, 40)
    nu = syn.gaussian_mixture(32, 4, 41)
    sched = syn.paper_schedule(32, 2, 5)
    total = sum(s[1] for s in sched)
    for cut in (3, total - 2):
        path = str(tmp_path / f"ckpt_{mode}_{cut}.bin")
        g = lib.DD(mu, nu, 4, 2, sched, err_tol=1e-6, mode=mode)
        g.sweep(cut)
        g.save(path)
        g.sweep(total - cut + 2)
        ref = _state(g)
        g.close()
        h = lib.DD.load(path)
        assert h.info()[0] == (0 if cut == 3 else 1)
        h.sweep(total - cut + 2)
        _assert_same_state(_state(h), ref)
        h.close()


def test_safeguard_rescues_every_forced_failure(lib):
    # debug_flags bit 3: every cell's main solve stops after one iteration;
    # the safeguard re-solves each at 4ε, then at ε, and the run ends at the
    # oracle's fixed point with no cell left at max_iter
    mu = syn.gaussian_mixture(32, 3, 50)
    nu = syn.gaussian_mixture(32, 3, 51)
    sched = WARM_SCHEDULE
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-6, max_iter=5000, debug_flags=8)
    st = g.run_schedule(strict=True)
    prof = g.profile()
    rp, col, val = g.basic_marginals()
    cost, _, ey = g.cost()
    g.close()
    ncells = (32 // 8) ** 2 + (32 // 8 + 1) ** 2
    assert st.cells_not_converged == 0
    assert st.cells_rescued > 0 and prof.rescued_cells >= ncells
    assert prof.sinkhorn_iters > prof.cells   # the re-solves iterate beyond the cut-off
    ref = odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))
    got = odd.rows_to_dense(odd.rows_from_csr(rp, col, val), 32 * 32)
    want = odd.rows_to_dense(ref.rows, 32 * 32)
    assert np.abs(got - want).sum() / want.sum() < PLAN_TOL
    assert abs(cost - ref.history[-1][3].cost) / ref.history[-1][3].cost < COST_TOL
    assert ey < 1e-10          # only the mass that Truncate dropped (≤ 1e-15 per entry)


def test_cells_at_max_iter_are_reported(lib):
    # with the safeguard off and one iteration per solve, the sweep completes
    # (a feasible state: the Y-marginal is exact) and reports the cells
    mu = syn.gaussian_mixture(32, 3, 52)
    nu = syn.gaussian_mixture(32, 3, 53)
    g = lib.DD(mu, nu, 4, 1, [(0.004, 2, 0)], err_tol=1e-7, max_iter=1, safeguard=0)
    with pytest.raises(lib.DDNotConverged) as e:
        g.sweep(1, strict=True)
    assert e.value.status == lib.DD_ERR_NOT_CONVERGED
    assert e.value.stats.cells_not_converged > 0 and e.value.stats.sweeps_done == 1
    _, _, ey = g.cost()
    assert ey < 1e-12
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        st = g.sweep(1)                     # default: a warning and the statistics
    assert any(issubclass(x.category, lib.DDConvergenceWarning) for x in w)
    assert st.sweeps_done == 2
    g.close()


def test_graph_overflow_reruns_with_per_kernel_launches(lib):
    # debug_flags bit 2: each graph-replayed sweep gets an output buffer of
    # half the entries, overflows, and is run again per kernel (from the duals
    # the graph's solves already updated, so the trajectory differs from the
    # per-kernel mode's within the solve tolerance); the input state must
    # survive the overflow intact: the run reaches the oracle's state
    mu = syn.gaussian_mixture(32, 3, 54)
    nu = syn.gaussian_mixture(32, 3, 55)
    sched = WARM_SCHEDULE + [(0.00625, 3, 0)]
    out = {}
    for mode, flags in ((0, 0), (1, 4)):
        g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-6, max_iter=5000, mode=mode, debug_flags=flags)
        g.run_schedule(strict=True)
        rp, col, val = g.basic_marginals()
        cost, _, ey = g.cost()
        out[mode] = (odd.rows_to_dense(odd.rows_from_csr(rp, col, val), 32 * 32), cost, ey, g.profile())
        g.close()
    assert out[1][3].graph_reruns > 0 and out[0][3].graph_reruns == 0
    ref = odd.run_schedule(mu, nu, 4, 1, sched, odd.Params(err=1e-10))
    want = odd.rows_to_dense(ref.rows, 32 * 32)
    ref_cost = ref.history[-1][3].cost
    for mode in (0, 1):
        got, cost, ey, _ = out[mode]
        assert np.abs(got - want).sum() / want.sum() < PLAN_TOL, mode
        assert abs(cost - ref_cost) / ref_cost < COST_TOL, mode
        assert ey < 1e-10, mode


def test_injected_workspace_allocation_failure(lib):
    # debug_flags bit 4: the first workspace allocation fails (DD_ERR_OOM)
    # before the state is touched; the next call runs, and the run reaches
    # the state of a run without the failure, bit for bit
    mu = syn.gaussian_mixture(32, 3, 56)
    nu = syn.gaussian_mixture(32, 3, 57)
    sched = WARM_SCHEDULE
    g = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-6, max_iter=5000, debug_flags=16)
    with pytest.raises(lib.DDError) as e:
        g.sweep(1)
    assert e.value.status == lib.DD_ERR_OOM and "injected" in str(e.value)
    g.run_schedule(strict=True)
    got = _state(g)
    g.close()
    r = lib.DD(mu, nu, 4, 1, sched, err_tol=1e-6, max_iter=5000)
    r.run_schedule(strict=True)
    _assert_same_state(got, _state(r))
    r.close()


def test_safeguard_escalates_epsilon_and_keeps_the_state_feasible(lib):
    # a cold start at a small ε with 50 iterations per solve: the main solves
    # and the re-solves at 4ε stop short, the safeguard goes on to 16ε, 64ε,
    # … and keeps the first solve that converges (status bit 3). Cells left
    # at max_iter are those the safeguard does not take: X-error at most
    # 10·Err·‖μ_J‖. The state stays feasible.
    n, b, err = 32, 4, 1e-6
    mu = syn.gaussian_mixture(n, 3, 58)
    nu = syn.gaussian_mixture(n, 3, 59)
    g = lib.DD(mu, nu, b, 1, [(0.002, 2, 0)], err_tol=err, max_iter=50)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        st = g.sweep(1)
    cs = g.cell_stats()
    prof = g.profile()
    _, ex, ey = g.cost()
    g.close()
    assert st.cells_escalated > 0
    assert int(((cs["status"] & 8) != 0).sum()) == st.cells_escalated
    assert prof.escalated_cells >= st.cells_escalated
    # ‖μ_J‖ of the B cells (the last half-sweep): basic cells 2a−1, 2a per axis
    m = mu / mu.sum()
    nb = n // b
    M = np.zeros((nb + 2, nb + 2))
    M[1:-1, 1:-1] = m.reshape(nb, b, nb, b).sum(axis=(1, 3))
    muJ = M.reshape(nb // 2 + 1, 2, nb // 2 + 1, 2).sum(axis=(1, 3)).reshape(-1)
    left = np.flatnonzero(cs["status"] & 1)
    assert left.size == st.cells_not_converged
    assert np.all(cs["err_x"][left] <= 10 * err * muJ[left] * (1 + 1e-6))
    assert np.all((cs["status"][cs["status"] & 8 != 0] & 7) == 0)
    assert ey < 1e-10
