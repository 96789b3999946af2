"""Runtime and iterations against the basic cell size s (the paper leaves the
choice of s open: §7.1 "Basic and composite partitions" fixes s = 4 for its
experiments, and the conclusion names the cell size as a question for later
work).

For every s the same synthetic image pair (1024×1024 by default, 8
anisotropic Gaussian blobs) runs the coarse-to-fine schedule of
`synthetic.paper_schedule` from a coarsest level of at least 8×8 pixels that
is a multiple of 2s, and then sweeps at the final ε = 2h² until both marginal
errors are ≤ 1e-6 and one sweep changes the transport cost by at most 1e-7
relative. Reported per s: wall time from host images to that point, sweeps
at the final ε, Sinkhorn iterations (total and per cell solve), Newton
steps, the final-level throughput (pixels·sweeps/s of the last sweeps, CUDA
events through the stream), stored entries and peak plan memory, and cells
the safeguard re-solved.

s = 16 (composite cells of 32×32 pixels) is beyond the cell solver, whose
cells hold at most 256 pixels in shared memory; it is reported as such.

    python -m paper_2001_10986_gb300.cell_size_study [--n 1024] [--sizes 2 4 8 16]
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import synthetic as syn


def levels_for(n: int, s: int) -> int:
    """Most levels whose coarsest side is ≥ 8 and a multiple of 2s."""
    best = 1
    for L in range(1, 16):
        n0 = n >> (L - 1)
        if n0 < 8 or n0 % (2 * s) or n % (1 << (L - 1)):
            break
        best = L
    return best


def run_one(n: int, s: int, workload: str = "gm1024_b4", err: float = 1e-6, max_final: int = 200,
            mode: int = 1, stream=None) -> dict:
    import torch
    from . import dd
    if 2 * s * 2 * s > 256:
        return {"s": s, "supported": False,
                "reason": "composite cells of (2s)² > 256 pixels exceed the cell solver's shared-memory layout"}
    w = syn.WORKLOADS[workload]
    mu, nu = syn.image_pair(w, 0)
    if mu.shape[0] != n:
        mu = syn.gaussian_mixture(n, w.blobs, 0, anisotropic=w.anisotropic, floor=w.floor)
        nu = syn.gaussian_mixture(n, w.blobs, 1, anisotropic=w.anisotropic, floor=w.floor)
    L = levels_for(n, s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = dd.DD(mu, nu, s, L, syn.paper_schedule(n, L, 1), err_tol=err, mode=mode, stream=stream)
    g.run_schedule()
    k, prev, done = 1, None, False
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    last_ms = []
    while k < max_final:
        cost, ex, ey = g.cost()
        rel = abs(cost - prev) / abs(cost) if prev is not None else math.inf
        prev = cost
        if ex <= 1e-6 and ey <= 1e-6 and rel <= 1e-7:
            done = True
            break
        ev0.record(torch.cuda.current_stream() if stream is None else stream)
        g.sweep(1)
        ev1.record(torch.cuda.current_stream() if stream is None else stream)
        torch.cuda.synchronize()
        last_ms.append(ev0.elapsed_time(ev1))
        k += 1
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    p = g.profile()
    _, _, nbasic, eps, nnz = g.info()
    g.close()
    tail = last_ms[-3:] if last_ms else [float("nan")]
    return {"s": s, "supported": True, "levels": L, "seconds_to_converged": seconds, "converged": done,
            "final_sweeps": k, "cost": cost, "err_x": ex, "err_y": ey,
            "sinkhorn_iters": p.sinkhorn_iters, "cell_solves": p.cells,
            "iters_per_cell_solve": p.sinkhorn_iters / max(p.cells, 1), "newton_steps": p.newton_steps,
            "final_level_px_sweeps_per_s": n * n / (sum(tail) / len(tail) * 1e-3),
            "entries_final": nnz, "peak_entries": p.peak_nnz, "peak_state_bytes": p.peak_state_bytes,
            "peak_work_bytes": p.peak_work_bytes, "rescued_cells": p.rescued_cells}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--sizes", type=int, nargs="+", default=[2, 4, 8, 16])
    ap.add_argument("--mode", type=int, default=1)
    args = ap.parse_args(argv)
    for s in args.sizes:
        print(json.dumps(run_one(args.n, s, mode=args.mode)), flush=True)


if __name__ == "__main__":
    main()
