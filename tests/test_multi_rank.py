"""Replicas-only multi-GPU path of bench.py, exercised on CPU with two gloo ranks:
the max-over-ranks timing and the whole-job throughput (units of all ranks over the
slowest rank's time).  No data-path collective exists to test."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [2.0, 3.5][rank]                       # each rank's timed seconds for K = 4 steps
    tmax = bench.max_over_ranks(t, dist, "cpu")
    dist.barrier()
    q.put((rank, tmax, bench.job_throughput(4, world, tmax)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, thr in out:
        assert tmax == 3.5
        assert abs(thr - 8 / 3.5) < 1e-12
