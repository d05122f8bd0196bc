"""The benchmark's multi-rank host logic on CPU: two processes joined by a gloo process
group.  Each rank advances its own slab (weak scaling), and the only collective is the
max-over-ranks reduction of the timing.  No GPU is used."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    import bench
    import synthgen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # every rank reports its own time; all of them get the slowest
        t = bench.max_over_ranks(100.0 + 50.0 * rank, ws, "cpu")
        cells = synthgen.slab(side=8, key=bench.workload_key(rank))
        n_sum = bench.max_over_ranks(float(np.sum(cells["n"])), ws, "cpu")
        q.put((rank, t, float(np.sum(cells["n"])), n_sum, bench.job_throughput(cells["n"].size, ws, 5, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = 2
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, m0, v0), (r1, t1, s1, m1, v1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 150.0                      # the slowest rank's time on both
    assert s0 != s1                               # different slabs per rank
    assert m0 == m1 == max(s0, s1)
    assert v0 == v1 == pytest.approx(2 * 512 * 5 / 0.150)   # all ranks' cells over the slowest time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(1000, 1, 2, 100.0) == pytest.approx(20000.0)
    assert bench.workload_key(0) != bench.workload_key(1)
