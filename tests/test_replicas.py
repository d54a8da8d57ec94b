"""Host logic of the multi-GPU bench path (one replica per rank, weak
scaling): the slowest rank's time is taken over all ranks and the rate
counts the cell updates of all ranks.  Runs as two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 30.0][rank]
        m = bench.max_over_ranks(ms, world, torch.device("cpu"))
        rate = bench.whole_job_rate(1000, 4, m, world)
        q.put((rank, m, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, rate in out:
        assert m == 30.0
        assert rate == pytest.approx(2 * 1000 * 4 / 30e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, None) == 7.0
    assert bench.whole_job_rate(10, 2, 4.0, 1) == pytest.approx(5000.0)
