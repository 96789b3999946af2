"""The full form at scale: 2048×2048 Gaussian-mixture images (12 blobs, floor
1e-4), 4×4 basic cells, five levels 128² → 2048², ε down to 2h², FP32 cell
solves with FP64 global sums, persistent graph-replayed sweeps, and the peak
device memory of the sparse plan.

One run per dual refinement (0: cell-wise first-order refinement; 1: the
glued dual of §6.3 interpolated by §6.4 for the B cells) and, optionally,
with the learned warm start: the coarse-to-fine schedule of
`synthetic.paper_schedule` (one sweep at the final ε), then sweeps at the
final ε until both marginal L1 errors are ≤ 1e-6 and one sweep changes the
transport cost by at most 1e-7 relative. Reported per run: wall time from
host images, cells still at max_iter after the schedule and at the end,
cells the local safeguard of §7.3 re-solved (and kept at a larger ε),
Sinkhorn iterations and Newton steps, peak entries of (ν_i) and peak device
memory of its CSR buffers and of the half-sweep work buffers, final-level
sweep throughput, cost and marginal errors.

    python -m paper_2001_10986_gb300.full_form [--dual-refine 0 1] [--learned]
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import synthetic as syn


def run(dual_refine: int = 0, mlp=None, workload: str = "gm2048_b4_l5", err: float = 1e-6,
        max_final: int = 60, mode: int = 1, start_cells: float = 0.0) -> dict:
    """start_cells: the coarsest level starts at ε = 2·(start_cells·Δ₀)² and
    halves down to 2Δ₀² (synthetic.paper_schedule's eps_start; 0 keeps its
    default 2·(1/8)², which at a 128² coarsest level makes the first plans
    nearly dense)."""
    import torch
    from . import dd
    w = syn.WORKLOADS[workload]
    mu, nu = syn.image_pair(w, 0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d0 = 2.0 ** (w.levels - 1) / w.n
    sched = (syn.paper_schedule(w.n, w.levels, 1, eps_start=2.0 * (start_cells * d0) ** 2) if start_cells > 0
             else syn.paper_schedule(w.n, w.levels, 1))
    g = dd.DD(mu, nu, w.b, w.levels, sched, err_tol=err, mode=mode,
              dual_refine=dual_refine, warm=1 if mlp is not None else 0, stream=stream)
    if mlp is not None:
        g.attach_mlp(mlp)
    st = g.run_schedule()
    torch.cuda.synchronize()
    t_sched = time.perf_counter() - t0
    nc_sched = st.cells_not_converged
    p_sched = g.profile()
    k, prev, done = 1, None, False
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    while True:
        cost, ex, ey = g.cost()
        rel = abs(cost - prev) / abs(cost) if prev is not None else math.inf
        prev = cost
        if (ex <= 1e-6 and ey <= 1e-6 and rel <= 1e-7) or k >= max_final:
            done = ex <= 1e-6 and ey <= 1e-6 and rel <= 1e-7
            break
        ev0.record(stream)
        st = g.sweep(1)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        k += 1
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    p = g.profile()
    _, _, _, eps, nnz = g.info()
    g.close()
    tail = ms[-3:] if ms else [float("nan")]
    return {"workload": workload, "dual_refine": dual_refine, "learned": mlp is not None,
            "eps_start": sched[0][0], "schedule_steps": len(sched),
            "seconds_schedule": t_sched, "seconds_to_converged": seconds, "converged": done, "final_sweeps": k,
            "cells_not_converged_after_schedule": nc_sched, "cells_not_converged_last": st.cells_not_converged,
            "rescued_cells_schedule": p_sched.rescued_cells, "rescued_cells": p.rescued_cells,
            "escalated_cells": p.escalated_cells,
            "sinkhorn_iters": p.sinkhorn_iters, "newton_steps": p.newton_steps,
            "peak_entries": p.peak_nnz, "peak_state_bytes": p.peak_state_bytes,
            "peak_work_bytes": p.peak_work_bytes, "entries_final": nnz,
            "final_level_px_sweeps_per_s": w.n * w.n / (sum(tail) / len(tail) * 1e-3),
            "cost": cost, "err_x": ex, "err_y": ey, "eps": eps}


def train_network(stream=None):
    """The warm-start network of the benchmark: pairs logged from plain runs
    on three 256² pairs (5 blobs, 3 levels), 20 epochs of Adam."""
    import torch
    from . import learned
    fs, ts = [], []
    for k in range(3):
        m2 = syn.gaussian_mixture(256, 5, 1000 + 2 * k)
        n2 = syn.gaussian_mixture(256, 5, 1001 + 2 * k)
        f, tg = learned.log_pairs(m2, n2, 4, 3, syn.paper_schedule(256, 3, 4), min_level=1, stream=stream)
        fs.append(f)
        ts.append(tg)
    return learned.train((torch.cat(fs), torch.cat(ts)), epochs=20, batch=512, lr=1e-3)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dual-refine", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--workload", default="gm2048_b4_l5")
    ap.add_argument("--start-cells", type=float, default=0.0)
    ap.add_argument("--max-final", type=int, default=60)
    args = ap.parse_args(argv)
    net = train_network() if args.learned else None
    for dr in args.dual_refine:
        print(json.dumps(run(dr, workload=args.workload, start_cells=args.start_cells, max_final=args.max_final)),
              flush=True)
        if net is not None:
            print(json.dumps(run(dr, mlp=net, workload=args.workload, start_cells=args.start_cells,
                                 max_final=args.max_final)), flush=True)
    if net is not None:
        net.close()


if __name__ == "__main__":
    main()
