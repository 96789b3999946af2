"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
image pair, agree on the job's timed duration (the maximum over ranks) and
on the whole-job throughput (replicas only: no collective on the data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from paper_2001_10986_gb300 import synthetic as syn
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        ms = 10.0 * (rank + 1)                       # the ranks finish at different times
        ms_max = bench.replica_timing(ms, dist, "cpu")
        value = bench.whole_job_value(64, 5, w, ms_max)
        mu, nu = syn.image_pair("gm32_b4", r)        # every rank solves its own pair
        q.put((r, w, ms_max, value, float(mu[3, 4]), float(nu[5, 6])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, v0, m0, n0), (r1, w1, t1, v1, m1, n1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 20.0
    assert v0 == v1 == pytest.approx(2 * 64 * 64 * 5 / 0.020)
    assert m0 != m1 and n0 != n1
