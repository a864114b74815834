"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2).

Each rank works on its own copy of the workload (weak scaling) with no data
exchange; the only cross-rank steps are the barrier and the max of the timed
region, which this test drives with different per-rank times.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, torch.device("cpu"))
    value = bench.weak_scaling_value(1_000_000, 10, ms, world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 150.0  # the slowest rank
        assert value == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(42.0, torch.device("cpu")) == 42.0
    assert bench.weak_scaling_value(10, 2, 1000.0, 1) == pytest.approx(20 / 1e9)
