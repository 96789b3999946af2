#!/usr/bin/env python
"""Throughput of the domain-decomposition half-sweep path on GB300.

Metric: pixels·sweeps/s at the finest level of a coarse-to-fine run on
1024×1024 Gaussian-mixture images (4×4 basic cells, layers 8²→1024², final
ε = 2h²). One step = one sweep (half-sweep on partition A, then on B) over the
whole image. The state (basic marginals, duals, workspace) stays resident in
HBM between steps and is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

With N > 1 (torchrun, one process per GPU) every rank solves its own image
pair (pair index = rank): the problems are independent, so the scaling is weak
and no collective touches the data path; only the timing uses a barrier and a
max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixels·sweeps/s at 1024², plain DD"
UNIT = "px·sweeps/s"
# FP32 lanes per SM (FFMA per clock), SMs and the maximum SM clock of a GB300:
# the ALU peak the cell-solve kernels are reported against
FP32_LANES_PER_SM = 128
NUM_SM = 152
SM_MAX_MHZ = 2070.0
# algorithmic FP32 work of the cell solves:
#  * every kernel entry of every Y-iteration: 2 FMAs (Σ_x K̃u for s(y) and
#    Σ_y K̃v for the X-marginal);
#  * every Newton X-iteration: the symmetric 64×64 Hessian, 64·65/2 FMAs per
#    support point (the profile counts 64² per point).
FMA_PER_ENTRY = 2.0
HESS_SYM = 65.0 / 128.0
# DRAM bytes per launch of the per-CTA cell-solve kernel k_sinkhorn, from an
# ncu capture of the current kernel (dram__bytes_read.sum + write.sum over the
# last two finest-level sweeps at 512²: 63.5 and 51.8 MB for the A, 56.8 and
# 54.9 MB for the B half-sweeps, mean 56.8 MB) scaled by the 4× cell count to
# 1024²; the cluster kernel beside it is not included
SOLVE_TRAFFIC_BYTES = 4 * 56.8e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    p.add_argument("--workload", default="gm1024_b4")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-ttc", action="store_true", help="skip the time-to-converged runs")
    p.add_argument("--no-learned", action="store_true", help="skip the learned warm-start arm")
    p.add_argument("--err", type=float, default=1e-6)
    p.add_argument("--tpc", type=int, default=0, help="threads per cell solve (0: library choice)")
    p.add_argument("--clusters", type=int, default=-1, help="max cells solved by 8-CTA clusters (-1: library choice)")
    p.add_argument("--mode", type=int, default=1, help="0: per-kernel launches, 1: persistent solves + graph-replayed sweeps")
    p.add_argument("--autotune", type=int, default=1, help="1: pick threads per cell and cluster cells by dd_autotune first")
    p.add_argument("--newton", type=int, default=1, help="dd_options.x_newton (0: plain X-iterations only)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class OracleBlock:
    """The FP64 oracle on a bounded sample of the same workload, in the same
    warm steady state the GPU arm sweeps: a block of 16×16 basic cells
    (64×64 pixels, 64 A cells and the 49 B cells inside it) of the 1024²
    problem at the final ε = 2h², with ν and the basic marginals of a
    feasible synthetic state (`synthetic.feasible_state`). `warm_sweeps`
    untimed oracle sweeps of the block (A then B, from zero duals) bring its
    cells to warm starts; every timed step is one more sweep of the block.
    px·sweeps/s of the block needs no extrapolation (the unit is intensive).
    The cells of a half-sweep are independent (§6.1) and are split over a
    pool of `workers` processes (started with spawn), each running the
    oracle's own half_sweep on its cells; workers = 1 runs in-process."""

    MARGIN = 16          # pixels of Y around the block (the rows reach ≤ 13)

    def __init__(self, workload, workers=1, block=16, warm_sweeps=6, err=1e-6):
        import numpy as np
        from oracle import dd as odd
        from paper_2001_10986_gb300 import synthetic as syn
        self.np, self.odd = np, odd
        w = syn.WORKLOADS[workload]
        self.n, self.b, self.err = w.n, w.b, err
        mu, _ = syn.image_pair(w, 0)
        # the feasible state of a window around the block only (its rows are
        # those of the full image: each depends on its own basic cell alone)
        b0 = (self.n // self.b) // 2 - block // 2          # first basic cell of the block
        m = self.MARGIN
        self.p0 = b0 * self.b - m                           # window origin (pixels)
        side = block * self.b + 2 * m
        nu_full, rp, col, val = syn.feasible_state(mu, self.b, seed=7)
        win_mu = mu[self.p0:self.p0 + side, self.p0:self.p0 + side]
        win_nu = nu_full[self.p0:self.p0 + side, self.p0:self.p0 + side]
        self.prob = odd.GridProblem(win_mu, win_nu, self.b, 1.0 / self.n)
        nbw, nbf = side // self.b, self.n // self.b
        rows = []
        for R in range(nbw):
            for S in range(nbw):
                i = (self.p0 // self.b + R) * nbf + (self.p0 // self.b + S)
                c = col[rp[i]:rp[i + 1]].astype(np.int64)
                r_, c_ = np.divmod(c, self.n)
                r_, c_ = r_ - self.p0, c_ - self.p0
                ok = (r_ >= 0) & (r_ < side) & (c_ >= 0) & (c_ < side)
                rows.append(((r_[ok] * side + c_[ok]), val[rp[i]:rp[i + 1]][ok].astype(np.float64)))
        self.rows = rows
        blk = set(range(m // self.b, m // self.b + block))
        def inside(J):
            return all((i // nbw) in blk and (i % nbw) in blk for i in J)
        self.cells = {p: [k for k, J in enumerate(self.prob.parts[p]) if inside(J)] for p in "AB"}
        self.eps = 2.0 / self.n ** 2
        self.alpha = {"A": np.zeros(side * side), "B": np.zeros(side * side)}
        self.px = (block * self.b) ** 2
        self.workers = max(1, int(workers))
        self.pool = None
        if self.workers > 1:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(
                self.workers, initializer=_oracle_block_init, initargs=(win_mu, win_nu, self.b, 1.0 / self.n))
        self.iters = []
        for _ in range(warm_sweeps):
            self.sweep()

    def _half(self, part):
        odd = self.odd
        cells = self.cells[part]
        if self.pool is None:
            self.rows, info = odd.half_sweep(self.prob, part, self.rows, self.alpha[part], self.eps,
                                             odd.Params(err=self.err), cells=cells)
            return list(info.iters)
        k = self.workers
        chunks = [cells[s::k] for s in range(k) if cells[s::k]]
        tasks = []
        for ch in chunks:
            need = {i for jn in ch for i in self.prob.parts[part][jn]}
            tasks.append((part, {i: self.rows[i] for i in need}, self.alpha[part], self.eps, self.err, ch))
        its = []
        for rows_sub, alpha_sub, it in self.pool.map(_oracle_block_task, tasks):
            for i, r in rows_sub.items():
                self.rows[i] = r
            for X, a in alpha_sub:
                self.alpha[part][X] = a
            its += it
        return its

    def sweep(self):
        t = time.perf_counter()
        its = self._half("A") + self._half("B")
        self.iters = its
        return time.perf_counter() - t

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


_BLOCK = {}


def _oracle_block_init(mu, nu, b, spacing):
    from oracle import dd as odd
    _BLOCK["prob"] = odd.GridProblem(mu, nu, b, spacing)


def _oracle_block_task(task):
    # one worker's share of a block half-sweep: the oracle's half_sweep on a
    # subset of the cells; returns their new rows and α
    from oracle import dd as odd
    prob = _BLOCK["prob"]
    part, rows_sub, alpha, eps, err, cells = task
    rows = [None] * len(prob.basic)
    for i, r in rows_sub.items():
        rows[i] = r
    alpha = alpha.copy()
    new_rows, info = odd.half_sweep(prob, part, rows, alpha, eps, odd.Params(err=err), cells=cells)
    out_rows, out_alpha = {}, []
    for jn in cells:
        J = prob.parts[part][jn]
        for i in J:
            out_rows[i] = new_rows[i]
        X = prob.cell_points(J)
        out_alpha.append((X, alpha[X]))
    return out_rows, out_alpha, list(info.iters)


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_baseline(workload, steps=2):
    """The oracle, as it stands, on the block sample (see OracleBlock), on all
    host cores and on one; px·sweeps/s of the timed block sweeps."""
    import numpy as np
    out = {}
    for workers in (host_cores(), 1):
        blk = OracleBlock(workload, workers=workers)
        ts = [blk.sweep() for _ in range(steps)]
        out[workers] = (blk.px * steps / sum(ts), float(np.mean(blk.iters)), sum(ts), blk)
        blk.close()
    cores = host_cores()
    v, it, dt, blk = out[cores]
    v1, _, dt1, _ = out[1]
    sample = (f"FP64 oracle, {steps} timed sweeps (A+B) of a 64×64-pixel block (16×16 basic cells: "
              f"{len(blk.cells['A'])} A + {len(blk.cells['B'])} B cells) of the {blk.n}² problem at eps=2h², "
              f"warm: 6 untimed oracle sweeps of the block from a feasible synthetic state first; "
              f"mean {it:.1f} Sinkhorn iterations per cell solve (plain iteration, Err 1e-6); "
              f"{dt:.1f} s on {cores} processes; 1 process: {v1:.4g} px·sweeps/s ({dt1:.1f} s)")
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "value_1_core": v1, "mean_iters_per_cell": it}


def replica_timing(ms_local, pg, device):
    """The timed region's duration as the job sees it: the maximum over the
    ranks of each rank's own duration (ms); pg is torch.distributed or None."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if pg:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n, steps, world, ms_max):
    """px·sweeps/s of all replicas together: each rank sweeps its own n×n pair."""
    return world * n * n * steps / (ms_max * 1e-3)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2001_10986_gb300 import synthetic as syn
    w = syn.WORKLOADS[args.workload]
    cores = host_cores()
    blk = OracleBlock(args.workload, workers=cores)
    for _ in range(args.warmup):
        blk.sweep()
    ts = [blk.sweep() for _ in range(args.steps)]
    its = blk.iters
    blk.close()
    import numpy as np
    ms = 1e3 * sum(ts) / max(len(ts), 1)
    v = blk.px / (ms * 1e-3)
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"each step: one sweep (A+B) of a 64×64-pixel block of the {w.n}² problem at eps=2h² "
                    f"(16×16 basic cells, warm after 6 untimed sweeps from a feasible synthetic state), "
                    f"FP64 oracle on {cores} processes; mean {float(np.mean(its)):.1f} iterations per cell; "
                    f"ms_per_step is the measured time of one block sweep"}
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "n": w.n, "b": w.b, "levels": w.levels,
                      "eps_final": "2h^2", "sample": "64x64-pixel block"},
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_golden(workload):
    """The FP64 oracle's state of a workload after its schedule and a fixed
    number of final sweeps, if stored (written by tests/golden/oracle_state.py):
    (json dict, npz of sampled rows)."""
    import numpy as np
    base = os.path.join(GOLDEN, f"oracle_state_{workload}")
    if not os.path.exists(base + ".json"):
        return None
    with open(base + ".json") as f:
        return json.load(f), dict(np.load(base + ".npz"))


def sampled_rows_rel_l1(rp, col, val, npz):
    """Relative L1 distance of basic marginals (ν_i) to the stored rows."""
    import numpy as np
    ids, grp, gcol, gval = (npz[k] for k in ("row_ids", "row_ptr", "col", "val"))
    num = den = 0.0
    for k, i in enumerate(ids):
        ce, ve = gcol[grp[k]:grp[k + 1]], gval[grp[k]:grp[k + 1]]
        cg, vg = col[rp[i]:rp[i + 1]], val[rp[i]:rp[i + 1]]
        u = np.union1d(ce, cg)
        a_ = np.zeros(u.size)
        a_[np.searchsorted(u, cg)] = vg
        e = np.zeros(u.size)
        e[np.searchsorted(u, ce)] = ve
        num += np.abs(a_ - e).sum()
        den += e.sum()
    return float(num / den)


def time_to_converged(dd, syn, mu, nu, w, args, stream, max_final_sweeps=400, mlp=None, **opts):
    """Wall time from host images to a converged plan: dd_create, the whole
    coarse-to-fine schedule (one sweep at the final ε), then sweeps at the
    final ε until both marginal L1 errors are ≤ 1e-6 and one sweep changes the
    transport cost by at most 1e-7 relative. Each check is one dd_cost call (a
    device→host read per sweep)."""
    import torch
    n, b, L = w.n, w.b, w.levels
    torch.cuda.synchronize()
    t = time.perf_counter()
    h = dd.DD(mu, nu, b, L, syn.paper_schedule(n, L, 1), err_tol=args.err, stream=stream,
              threads_per_cell=args.tpc if w.n == 1024 else 0,
              max_cluster_cells=args.clusters if w.n == 1024 else -1, mode=args.mode, x_newton=args.newton, **opts)
    if mlp is not None:
        h.attach_mlp(mlp)
    h.run_schedule()
    k, rel, prev = 1, None, None
    while True:
        cost, ex, ey = h.cost()
        rel = abs(cost - prev) / abs(cost) if prev is not None else None
        done = ex <= 1e-6 and ey <= 1e-6 and rel is not None and rel <= 1e-7
        prev = cost
        if done or k >= max_final_sweeps:
            break
        h.sweep(1)
        k += 1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    p = h.profile()
    h.close()
    return {"seconds": dt, "final_sweeps": k, "converged": bool(done), "last_rel_change": rel, "cost": cost,
            "err_x": ex, "err_y": ey, "sinkhorn_iters": p.sinkhorn_iters, "newton_steps": p.newton_steps,
            "learned_cells": p.learned_cells, "compared_cells": p.compared_cells,
            "rescued_cells": p.rescued_cells, "peak_state_bytes": p.peak_state_bytes,
            "criterion": "err_x, err_y <= 1e-6 and relative cost change over one final-eps sweep <= 1e-7"}


def oracle_parity_256(dd, syn, args, stream, mlp=None, **opts):
    """The 256² workload's schedule and the stored oracle run's number of
    final sweeps on the GPU, timed from host images, then compared with the
    oracle's state (tests/golden): cost, marginal errors, sampled basic
    marginals."""
    import torch
    gold = load_golden("gm256_b4_l3")
    if gold is None:
        return None
    w = syn.WORKLOADS["gm256_b4_l3"]
    mu, nu = syn.image_pair(w, 0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    h = dd.DD(mu, nu, w.b, w.levels, syn.paper_schedule(w.n, w.levels, gold[0]["final_sweeps"]), err_tol=args.err,
              stream=stream, mode=args.mode, x_newton=args.newton, **opts)
    if mlp is not None:
        h.attach_mlp(mlp)
    h.run_schedule()
    cost, ex, ey = h.cost()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    rp, col, val = h.basic_marginals()
    p = h.profile()
    h.close()
    return {"seconds": dt, "cost": cost, "oracle_cost": gold[0]["cost"],
            "cost_rel": abs(cost - gold[0]["cost"]) / gold[0]["cost"], "err_x": ex, "err_y": ey,
            "plan_rel_l1": sampled_rows_rel_l1(rp, col, val, gold[1]),
            "plan_rows_compared": int(gold[1]["row_ids"].size), "sinkhorn_iters": p.sinkhorn_iters,
            "oracle_seconds": gold[0]["seconds"], "oracle_workers": gold[0]["workers"],
            "what": "same schedule and final sweeps as the stored FP64 oracle run; the oracle's wall time is "
                    "its own run on this build machine's cores"}


def run_cuda(args):
    import numpy as np
    import torch

    from paper_2001_10986_gb300 import build as bld
    if not os.path.exists(bld.LIB):
        bld.build()
    from paper_2001_10986_gb300 import dd, synthetic as syn

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = tdist
    w = syn.WORKLOADS[args.workload]
    n, b, L = w.n, w.b, w.levels
    mu, nu = syn.image_pair(w, rank)
    sched = syn.paper_schedule(n, L, args.warmup)
    stream = torch.cuda.current_stream()

    # ---- setup (untimed): coarse levels, refinement, warm-up sweeps at 2h² ----
    g = dd.DD(mu, nu, b, L, sched, err_tol=args.err, stream=stream, debug_flags=2 if args.mode == 0 else 0,
              threads_per_cell=args.tpc, max_cluster_cells=args.clusters, mode=args.mode,
              x_newton=args.newton)
    g.run_schedule()
    tuned = None
    if args.autotune:
        # untimed: 9 more sweeps at the final ε, one per launch-schedule candidate
        tuned = g.autotune(rounds=1)
        args.tpc, args.clusters = tuned
    torch.cuda.synchronize()
    g.reset_profile()
    lvl, nl, _, eps, nnz0 = g.info()
    assert nl == n, (nl, n)

    # ---- timed region: K sweeps at the finest level ----
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            st = g.sweep(1)
        e1.record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms_total = e0.elapsed_time(e1)
    prof = g.profile()
    cost, ex, ey = g.cost()
    g.close()
    if args.mode != 0:
        # kernel durations for the roofline: the same sweeps with per-kernel
        # launches and CUDA events (a graph replay has no per-kernel events)
        gk = dd.DD(mu, nu, b, L, sched, err_tol=args.err, stream=stream, debug_flags=2,
                   threads_per_cell=tuned[0] if tuned else args.tpc,
                   max_cluster_cells=tuned[1] if tuned else args.clusters, mode=0, x_newton=args.newton)
        gk.run_schedule()
        gk.reset_profile()
        for _ in range(min(args.steps, 3)):
            gk.sweep(1)
        torch.cuda.synchronize()
        prof_k = gk.profile()
        gk.close()
    else:
        prof_k = prof
    ms_max = replica_timing(ms_total, pg, "cuda")
    value = whole_job_value(n, args.steps, world, ms_max)

    # ---- roofline of the cell-solve kernels (FP32 ALU) ----
    launches = max(prof_k.solve_launches, 1)
    solve_ms = prof_k.solve_ms / launches
    fma = (FMA_PER_ENTRY * prof_k.kernel_evals + HESS_SYM * prof_k.hessian_fma) / launches
    achieved = 2.0 * fma / (solve_ms * 1e-3) / 1e12
    peak = NUM_SM * FP32_LANES_PER_SM * 2.0 * SM_MAX_MHZ * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": "k_sinkhorn + k_sinkhorn_cluster (one half-sweep's cell solves)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": SOLVE_TRAFFIC_BYTES, "traffic_kernel": "k_sinkhorn (per-CTA solves)",
                "peak_source": f"FP32 FMA: {NUM_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz "
                               "(unit counts and maximum clock)",
                "fma_per_launch": fma, "kernel_entries_per_launch": prof_k.kernel_evals / launches,
                "newton_steps_per_launch": prof_k.newton_steps / launches, "ms_per_launch": solve_ms,
                "solve_share_per_kernel_mode": prof_k.solve_ms / max(prof_k.half_sweeps, 1) * 2 / (ms_total / args.steps) if ms_total > 0 else None,
                "gather_ms_per_launch": prof_k.gather_ms / max(prof_k.gather_launches, 1),
                "cluster_ms_per_launch": prof_k.cluster_ms / launches,
                "mean_sinkhorn_iters": prof_k.sinkhorn_iters / max(prof_k.cells, 1)}

    # ---- end to end through the C ABI from host buffers ----
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t = time.perf_counter()
        sched_e2e = syn.paper_schedule(n, L, args.steps)
        h = dd.DD(mu, nu, b, L, sched_e2e, err_tol=args.err, stream=stream, threads_per_cell=args.tpc,
                  max_cluster_cells=args.clusters, mode=args.mode, x_newton=args.newton)
        h.run_schedule()
        c2, ex2_, ey2 = h.cost()
        rp, col, val = h.basic_marginals()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        h.close()
        e2e = {"value": n * n * args.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(2 * n * n * 8),
               "d2h_bytes_per_step": int(rp.nbytes + col.nbytes + val.nbytes + 24),
               "what": f"dd_create from host images + full schedule ({len(sched_e2e)} steps, "
                       f"{args.steps} sweeps at {n}²) + dd_cost + basic marginals to host; "
                       f"px·sweeps over the finest-level sweeps / wall time",
               "seconds": dt}

    ttc = None
    par256 = None
    if not args.no_ttc:
        ttc = {"plain": time_to_converged(dd, syn, mu, nu, w, args, stream)}
        # the hybrid refinement: B cells of each new level start from the
        # glued coarse dual (§6.3) interpolated linearly (§6.4), on the GPU
        ttc["glued_refinement"] = time_to_converged(dd, syn, mu, nu, w, args, stream, dual_refine=1)
        par256 = {"plain": oracle_parity_256(dd, syn, args, stream)}
        if not args.no_learned:
            # learned warm start: network trained on pairs logged from plain
            # runs on 256² images (5 blobs, 3 levels), compared cell by cell
            from paper_2001_10986_gb300 import learned
            import torch
            t0 = time.perf_counter()
            fs, ts = [], []
            for k in range(3):
                m2 = syn.gaussian_mixture(256, 5, 1000 + 2 * k)
                n2 = syn.gaussian_mixture(256, 5, 1001 + 2 * k)
                f, tg = learned.log_pairs(m2, n2, 4, 3, syn.paper_schedule(256, 3, 4), min_level=1,
                                          stream=stream)
                fs.append(f)
                ts.append(tg)
            net = learned.train((torch.cat(fs), torch.cat(ts)), epochs=20, batch=512, lr=1e-3)
            torch.cuda.synchronize()
            t_train = time.perf_counter() - t0
            for mode in (1, 2):
                res = time_to_converged(dd, syn, mu, nu, w, args, stream, warm=mode, mlp=net)
                res["training_seconds"] = t_train
                res["training_pairs"] = int(sum(x.shape[0] for x in fs))
                res["warm"] = mode
                ttc["learned" if mode == 1 else "learned_every_eps"] = res
            if par256["plain"] is not None:
                par256["learned"] = oracle_parity_256(dd, syn, args, stream, mlp=net, warm=1)
            # the evaluation case of the learned warm start: 512², 6 blobs, the
            # whole schedule with the previous duals and with the prediction
            ev = {}
            w5 = syn.WORKLOADS["gm512_b4"]
            m5, n5 = syn.image_pair(w5, 0)
            for mode in (0, 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = dd.DD(m5, n5, w5.b, w5.levels, syn.paper_schedule(w5.n, w5.levels, 3), err_tol=args.err,
                          stream=stream, warm=mode, mode=args.mode, x_newton=args.newton)
                if mode:
                    h.attach_mlp(net)
                h.run_schedule()
                c5 = h.cost(with_y=False)[0]
                torch.cuda.synchronize()
                p5 = h.profile()
                ev["learned" if mode else "previous_duals"] = {
                    "seconds": time.perf_counter() - t0, "sinkhorn_iters": p5.sinkhorn_iters,
                    "newton_steps": p5.newton_steps, "learned_cells": p5.learned_cells,
                    "compared_cells": p5.compared_cells, "cost": c5}
                h.close()
            ttc["learned_eval_gm512_b4"] = ev
            net.close()

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(args.workload)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "n": n, "b": b, "levels": L, "eps_final": eps,
                      "err_tol": args.err, "nnz": nnz0, "l2": "working set larger than L2 (CSR + workspace)",
                      "parallelism": f"replicas x{world} (independent image pairs)",
                      "mode": "persistent solves + graph-replayed sweeps" if args.mode == 1 else "per-kernel launches",
                      "autotuned": None if tuned is None else {"threads_per_cell": tuned[0],
                                                                "max_cluster_cells": tuned[1]}},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "time_to_converged": ttc,
           "oracle_parity_gm256_b4_l3": par256,
           "gpu_launches": int(prof.launches), "clocks": clk.summary(),
           "quality": {"cost": cost, "err_x": ex, "err_y": ey, "max_iters_last": st.max_iters,
                       "mean_iters_last": st.mean_iters, "cells_not_converged_last": st.cells_not_converged}}
    print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
