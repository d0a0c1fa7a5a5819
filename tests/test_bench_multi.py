"""The benchmark's N > 1 path on CPU: two gloo ranks, each a replica with its own timed
region; rank 0 reports N x steps / (slowest rank's time)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        worst = bench.max_over_ranks(times[rank], world, "cpu")
        out.put((rank, worst, bench.replica_rate(world, 20, worst)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.5, 0.8]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, rate in res:
        assert worst == 0.8  # every rank sees the slowest replica
        assert rate == pytest.approx(2 * 20 / 0.8)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.replica_rate(1, 10, 2.0) == 5.0
