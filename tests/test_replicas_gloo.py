"""The N > 1 path of bench.py on CPU: two ranks of a gloo process group.

The benchmark runs independent replicas (the H^2 apply does not shard): each
rank times its own apply, the job's time is the slowest rank's (all-reduce
MAX), and the whole-job throughput counts the units of every rank over that
time.  Two spawned processes check the reduction and the throughput they
report, and that a failing rank is seen by the parent (no hang).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out, fail_rank):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        if rank == fail_rank:
            raise RuntimeError("planted failure")
        per_rank_s = [0.5, 0.8][rank]  # the second replica is slower
        t = bench.max_over_ranks(per_rank_s, world, "cpu")
        out[rank] = (t, bench.replica_throughput(1000.0, t, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_max_time_and_throughput():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out, -1), nprocs=2, join=True, start_method="spawn")
        for r in range(2):
            t, value = out[r]
            assert t == 0.8  # the slowest replica sets the job's time
            assert value == pytest.approx(2 * 1000.0 / 0.8)


@pytest.mark.timeout(120)
def test_failing_rank_is_reported():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        with pytest.raises(Exception):
            mp.start_processes(_rank, args=(2, _free_port(), out, 1), nprocs=2, join=True, start_method="spawn")
