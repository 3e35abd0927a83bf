"""The benchmark's multi-rank plumbing on CPU: two gloo ranks, each with its
own timing, agree on the slowest rank's time and the whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [100.0 + 50.0 * rank, 7.0 - rank]  # total ms, e2e s
    total_ms, e2e = bench.max_over_ranks(mine, dist)
    out[rank] = (total_ms, e2e, bench.job_throughput(world, 4, 1000, total_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        total_ms, e2e, tput = out[r]
        assert total_ms == 150.0 and e2e == 7.0
        assert tput == pytest.approx(2 * 4 * 1000 / 0.150)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_throughput(1, 10, 5.0, 1000.0) == 50.0
