"""FP64 oracle states of full-size workloads after a fixed number of sweeps,
stored for the GPU parity tests and the benchmark.

This script calls only the FP64 oracle (`oracle/`) and the seeded image
generators (`paper_2001_10986_gb300/synthetic.py`, no method arithmetic). It
runs Algorithm 2 (§6.1) inside the multi-scale / ε-scaling driver of §6.4 —
the schedule the library's benchmark uses (`synthetic.paper_schedule`, one
sweep at the final ε = 2h²) — and then `--final-sweeps` more sweeps at the
final ε (or, with `--tol`, until one sweep changes the transport cost by at
most that much relative; at 256² and ε = 2h² the iteration contracts slowly,
about 5 % of the cost change per sweep, so the fixed point itself is out of
reach of this oracle's run time).

The composite cells of one half-sweep are independent (§6.1), so a pool of
worker processes (started with `spawn`) splits them: every worker runs the
oracle's own `half_sweep` on a subset of the cells, unchanged, and the
results are merged (new basic marginals of the cells' basic cells, α on their
pixels, cost / X-error / iteration sums). The dual refinement is the oracle's
cell-wise reading (`refine_duals`), the library's default.

Output, next to this file:
  oracle_state_<workload>.json  cost, marginal errors, the per-sweep cost at
                                the final ε, iteration counts, wall times,
                                cores used, the sweeps run;
  oracle_state_<workload>.npz   a seeded sample of basic rows of the final
                                state (row ids, CSR of those rows), for plan
                                comparisons.

  python tests/golden/oracle_state.py gm256_b4_l3 [--workers N] [--err 1e-8] [--final-sweeps 2]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import dd as odd  # noqa: E402
from paper_2001_10986_gb300 import synthetic as syn  # noqa: E402

# basic rows kept in the .npz per workload (seeded choice)
SAMPLE_ROWS = 512

_W = {}   # worker cache: level → GridProblem


def _init_worker(workload, levels):
    w = syn.WORKLOADS[workload]
    mu, nu = syn.image_pair(w, 0)
    _W["pyr"] = (odd.pyramid(mu / mu.sum(), levels), odd.pyramid(nu / nu.sum(), levels))
    _W["meta"] = (w.n, w.b, levels)
    _W["probs"] = {}


def _level_problem(lev):
    if lev not in _W["probs"]:
        n, b, levels = _W["meta"]
        mus, nus = _W["pyr"]
        _W["probs"] = {lev: odd.GridProblem(mus[lev], nus[lev], b, 2.0 ** (levels - 1 - lev) / n)}
    return _W["probs"][lev]


def _solve_chunk(task):
    lev, part, cells, rows_sub, alpha, eps, err, max_iter = task
    prob = _level_problem(lev)
    rows = [None] * len(prob.basic)
    for i, r in rows_sub.items():
        rows[i] = r
    alpha = alpha.copy()
    new_rows, info = odd.half_sweep(prob, part, rows, alpha, eps, odd.Params(err=err, max_iter=max_iter),
                                    cells=cells)
    out_rows, out_alpha = {}, {}
    for jn in cells:
        J = prob.parts[part][jn]
        for i in J:
            out_rows[i] = new_rows[i]
        X = prob.cell_points(J)
        out_alpha[jn] = (X, alpha[X])
    return out_rows, out_alpha, info.cost, info.err_x, list(info.iters), info.truncated_mass


def _chunks(ncells, k):
    # interleaved chunks: neighbouring cells (similar cost) go to different chunks
    return [list(range(s, ncells, k)) for s in range(k) if s < ncells]


def parallel_half_sweep(pool, prob, lev, part, rows, alpha, eps, err, max_iter, nchunks):
    cells_all = prob.parts[part]
    tasks = []
    for cells in _chunks(len(cells_all), nchunks):
        need = {i for jn in cells for i in cells_all[jn]}
        tasks.append((lev, part, cells, {i: rows[i] for i in need}, alpha, eps, err, max_iter))
    new_rows = list(rows)
    cost = errx = trunc = 0.0
    iters = []
    for out_rows, out_alpha, c, e, it, tm in pool.imap_unordered(_solve_chunk, tasks):
        for i, r in out_rows.items():
            new_rows[i] = r
        for X, a in out_alpha.values():
            alpha[X] = a
        cost += c
        errx += e
        iters += it
        trunc += tm
    return new_rows, cost, errx, iters, trunc


def converge(workload, workers, err, tol, max_final, max_iter, log=print):
    """The schedule, then sweeps at the final ε: max_final − 1 of them, or
    fewer once one sweep changes the cost by at most tol relative (tol > 0)."""
    w = syn.WORKLOADS[workload]
    n, b, levels = w.n, w.b, w.levels
    sched = syn.paper_schedule(n, levels, 1)
    mu, nu = syn.image_pair(w, 0)
    mus, nus = odd.pyramid(mu / mu.sum(), levels), odd.pyramid(nu / nu.sum(), levels)

    def level_problem(l):
        return odd.GridProblem(mus[l], nus[l], b, 2.0 ** (levels - 1 - l) / n)

    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    history = []
    with ctx.Pool(workers, initializer=_init_worker, initargs=(workload, levels)) as pool:
        lev = 0
        prob = level_problem(0)
        rows = odd.product_state(prob)
        alpha = {"A": np.zeros(prob.mu.size), "B": np.zeros(prob.mu.size)}
        last = "B"
        nchunks = 4 * workers
        total_iters = 0

        def sweep(eps):
            nonlocal rows, last, total_iters
            res = None
            for part in ("A", "B"):
                rows, cost, errx, iters, trunc = parallel_half_sweep(
                    pool, prob, lev, part, rows, alpha[part], eps, err, max_iter, nchunks)
                last = part
                total_iters += int(np.sum(iters))
                res = (cost, errx, int(np.max(iters)), float(np.mean(iters)), trunc)
            return res

        for eps_s, sweeps, L in sched:
            while lev < L:
                fine = level_problem(lev + 1)
                rows = odd.refine_basic_marginals(prob, fine, rows)
                a0 = odd.refine_duals(prob, fine, alpha[last], last)
                alpha = {"A": a0.copy(), "B": a0.copy()}
                prob, lev = fine, lev + 1
            for _ in range(sweeps):
                cost, errx, imax, imean, _ = sweep(eps_s)
                log(f"level {lev} eps {eps_s:.3e} cost {cost:.12e} err_x {errx:.2e} iters max {imax} "
                    f"mean {imean:.1f}  t={time.perf_counter() - t0:.0f}s")
        t_sched = time.perf_counter() - t0
        eps = sched[-1][0]
        prev = cost
        history.append(cost)
        k, rel, trunc = 1, None, 0.0
        while k < max_final:
            cost, errx, imax, imean, trunc = sweep(eps)
            k += 1
            history.append(cost)
            rel = abs(cost - prev) / abs(cost)
            prev = cost
            log(f"final sweep {k}: cost {cost:.15e} rel change {rel:.2e} err_x {errx:.2e} iters max {imax} "
                f"mean {imean:.1f}  t={time.perf_counter() - t0:.0f}s")
            if tol > 0 and rel <= tol:
                break
    t_all = time.perf_counter() - t0
    err_y = odd.y_marginal_error(prob, rows)
    return dict(workload=workload, n=n, b=b, levels=levels, eps=eps, oracle_err=err, tol=tol,
                cost=cost, err_x=errx, err_y=err_y, last_rel_change=rel, final_sweeps=k,
                final_costs=history, truncated_mass_last=trunc, sinkhorn_iters=total_iters,
                seconds_schedule=t_sched, seconds=t_all, workers=workers, nnz=int(sum(len(c) for c, _ in rows)),
                schedule="synthetic.paper_schedule(n, levels, 1), then final_sweeps - 1 more sweeps at the final eps"), rows


def save(res, rows, path_base):
    rng = np.random.default_rng(12345)
    nrows = len(rows)
    ids = np.sort(rng.choice(nrows, min(SAMPLE_ROWS, nrows), replace=False)).astype(np.int64)
    rp = np.zeros(ids.size + 1, dtype=np.int64)
    cols, vals = [], []
    for k, i in enumerate(ids):
        c, v = rows[i]
        rp[k + 1] = rp[k] + c.size
        cols.append(np.asarray(c, dtype=np.int32))
        vals.append(np.asarray(v, dtype=np.float64))
    np.savez_compressed(path_base + ".npz", row_ids=ids, row_ptr=rp, col=np.concatenate(cols),
                        val=np.concatenate(vals))
    res = dict(res)
    res["sample_rows"] = int(ids.size)
    with open(path_base + ".json", "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")


def main():
    p = argparse.ArgumentParser()
    p.add_argument("workload")
    p.add_argument("--workers", type=int, default=len(os.sched_getaffinity(0)))
    p.add_argument("--err", type=float, default=1e-8)
    p.add_argument("--tol", type=float, default=0.0)
    p.add_argument("--final-sweeps", type=int, default=2, help="sweeps at the final eps after the schedule's one")
    p.add_argument("--max-iter", type=int, default=100000)
    a = p.parse_args()
    res, rows = converge(a.workload, a.workers, a.err, a.tol, a.final_sweeps + 1, a.max_iter,
                         log=lambda s: print(s, flush=True))
    save(res, rows, os.path.join(HERE, f"oracle_state_{a.workload}"))
    print(json.dumps({k: v for k, v in res.items() if k != "final_costs"}))


if __name__ == "__main__":
    main()
