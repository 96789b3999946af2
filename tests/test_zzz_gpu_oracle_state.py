"""The full coarse-to-fine GPU run of the 256² workload (5 blobs, 4×4 basic
cells, 64² → 128² → 256², final ε = 2h²) against the FP64 oracle's run of the
same schedule and the same number of final sweeps, stored in
tests/golden/oracle_state_gm256_b4_l3.{json,npz} (written by
tests/golden/oracle_state.py, which calls only the oracle; the oracle takes
tens of minutes on eight cores, far beyond a test).

After the same sweeps, the GPU state must match the oracle's: transport cost
within 1e-6 relative, X- and Y-marginal errors ≤ 1e-6 in L1, and the basic
marginals (ν_i) within 1e-5 relative L1 on the stored sample of basic cells.
"""
import json
import os

import numpy as np
import pytest

from paper_2001_10986_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_state_gm256_b4_l3")
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


def sampled_rows_rel_l1(rp, col, val, gold_npz):
    """Relative L1 distance of the basic marginals (ν_i) on the stored rows."""
    ids, grp, gcol, gval = (gold_npz[k] for k in ("row_ids", "row_ptr", "col", "val"))
    num = den = 0.0
    for k, i in enumerate(ids):
        ce, ve = gcol[grp[k]:grp[k + 1]], gval[grp[k]:grp[k + 1]]
        cg, vg = col[rp[i]:rp[i + 1]], val[rp[i]:rp[i + 1]]
        u = np.union1d(ce, cg)
        a = np.zeros(u.size)
        a[np.searchsorted(u, cg)] = vg
        e = np.zeros(u.size)
        e[np.searchsorted(u, ce)] = ve
        num += np.abs(a - e).sum()
        den += e.sum()
    return num / den


@pytest.mark.skipif(not os.path.exists(GOLD + ".json"), reason="oracle state not stored")
@pytest.mark.parametrize("mode", [1, 0])
def test_gm256_full_schedule_matches_the_oracle(lib, mode):
    gold = json.load(open(GOLD + ".json"))
    npz = np.load(GOLD + ".npz")
    w = syn.WORKLOADS["gm256_b4_l3"]
    mu, nu = syn.image_pair(w, 0)
    g = lib.DD(mu, nu, w.b, w.levels, syn.paper_schedule(w.n, w.levels, gold["final_sweeps"]), err_tol=1e-6,
               mode=mode)
    g.run_schedule()
    cost, ex, ey = g.cost()
    rp, col, val = g.basic_marginals()
    _, nl, _, eps, _ = g.info()
    g.close()
    assert nl == w.n and eps == pytest.approx(gold["eps"], rel=1e-12)
    assert abs(cost - gold["cost"]) / gold["cost"] < COST_TOL, (cost, gold["cost"])
    assert ex < MARG_TOL and ey < MARG_TOL, (ex, ey)
    assert sampled_rows_rel_l1(rp, col, val, npz) < PLAN_TOL
