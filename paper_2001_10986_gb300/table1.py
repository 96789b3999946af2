"""The quantities of the paper's Table 1 (§7.1–7.3) for runs of this library.

One run follows the paper's iteration protocol (`synthetic.table1_schedule`:
per layer 2 sweeps at 2Δ², 1 at Δ², 1 at Δ²/2 from 8×8 up, 1 more at Δ²/4 on
the finest layer) with the paper's stopping criterion Err = 1e-4 on a pair
of synthetic Gaussian mixtures, and reports the rows of the table:

* total runtime (wall clock from host images to the last sweep, one GPU);
* entries of (ν_i): the maximum on the finest layer (at its largest ε) and
  the final number;
* relative primal-dual gap of eq. RelPDGap (glued duals and gap on the GPU,
  `DD.relative_pd_gap`; with --host-gap also the host evaluation of the same
  state, and both times);
* L1 marginal errors of X and Y (`dd_cost`);
* beside the table: peak device memory of the sparse plan and the cells that
  the local safeguard of §7.3 re-solved.

Usage (on a machine with a GPU):

    python -m paper_2001_10986_gb300.table1 64 128 256 --pairs 3

prints one JSON line per image size with the mean and standard deviation over
the pairs, in Table 1's units. The paper's images are not available, so the
numbers are comparable in magnitude only.
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import numpy as np

from . import synthetic as syn


def run_one(n: int, pair: int, *, blobs: int = 6, floor: float = 1e-4, b: int = 4, err: float = 1e-4,
            host_gap: bool = False, **opts) -> dict:
    from . import dd
    mu = syn.gaussian_mixture(n, blobs, 2 * pair, floor=floor)
    nu = syn.gaussian_mixture(n, blobs, 2 * pair + 1, floor=floor)
    sched, levels = syn.table1_schedule(n)
    total = sum(s for _, s, _ in sched)
    t0 = time.perf_counter()
    g = dd.DD(mu, nu, b, levels, sched, err_tol=err, **opts)
    try:
        nnz_max_finest = 0
        nnz_final = 0
        for _ in range(total):
            st = g.sweep(1)
            if st.level == levels - 1:
                nnz_max_finest = max(nnz_max_finest, int(st.nnz))
            nnz_final = int(st.nnz)
        seconds = time.perf_counter() - t0
        _, err_x, err_y = g.cost()
        t1 = time.perf_counter()
        rel, _, _ = g.relative_pd_gap()
        gap_s = time.perf_counter() - t1
        extra = {}
        if host_gap:
            t1 = time.perf_counter()
            extra["relative_pd_gap_host"] = g.relative_pd_gap(mu, nu, device=False)[0]
            extra["gap_host_s"] = time.perf_counter() - t1
        prof = g.profile()
    finally:
        g.close()
    return {"time_s": seconds, "entries_max": nnz_max_finest, "entries_final": nnz_final,
            "relative_pd_gap": rel, "gap_s": gap_s, "l1_error_x": err_x, "l1_error_y": err_y,
            "peak_state_bytes": prof.peak_state_bytes, "safeguard_cells": prof.rescued_cells, **extra}


def _mean_std(xs):
    return [statistics.fmean(xs), statistics.pstdev(xs) if len(xs) > 1 else 0.0]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("sizes", type=int, nargs="+", help="image sides (powers of two, ≥ 16)")
    ap.add_argument("--pairs", type=int, default=3)
    ap.add_argument("--blobs", type=int, default=6)
    ap.add_argument("--mode", type=int, default=1)
    ap.add_argument("--dual-refine", type=int, default=0)
    ap.add_argument("--host-gap", action="store_true")
    args = ap.parse_args(argv)
    for n in args.sizes:
        runs = [run_one(n, k, blobs=args.blobs, mode=args.mode, dual_refine=args.dual_refine,
                        host_gap=args.host_gap)
                for k in range(args.pairs)]
        out = {"image_size": n, "pairs": args.pairs, "iterations": (int(np.log2(n)) - 2) * 8 + 2}
        for key in runs[0]:
            out[key] = _mean_std([r[key] for r in runs])
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
