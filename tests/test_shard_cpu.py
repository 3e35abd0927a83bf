"""Rotation sharding on CPU: the shard ranges, the combine rule (the
kernels' argmin order over (cost, rotation index)) and the gloo all-gather of
result structs between two ranks. No GPU: dses_shard_range and
dses_combine_results are host functions of the C ABI library."""
import math
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2502_00115_b300 import build as b
from paper_2502_00115_b300 import capi


@pytest.fixture(scope="module", autouse=True)
def lib():
    b.build()
    return capi.load()


def res(cost, index, status=capi.DSES_OK, inliers=0):
    r = capi.dses_result()
    r.cost = cost
    r.rot_index = index
    r.status = status
    r.inliers = inliers
    r.t[:] = [float(index), 0.0, 0.0]
    return r


@pytest.mark.parametrize("n,world", [(72, 1), (72, 5), (294912, 8), (3, 7), (0, 3)])
def test_shard_ranges_tile_the_grid(n, world):
    ranges = [capi.shard_range(n, k, world) for k in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def test_shard_range_rejects_bad_arguments():
    for n, k, w in ((10, -1, 2), (10, 2, 2), (10, 0, 0), (-1, 0, 1)):
        st, _, _ = capi.dses_shard_range(n, k, w)
        assert st == capi.DSES_ERR_INVALID_ARG


def test_combine_takes_the_argmin_order():
    # lowest cost wins; equal costs go to the smaller rotation index
    parts = [res(0.5, 40), res(0.25, 900), res(0.25, 7), res(1.0, 3)]
    out = capi.combine_results(parts)
    assert out.rot_index == 7 and out.cost == 0.25 and out.status == capi.DSES_OK
    assert out.t[0] == 7.0
    # order of the parts does not matter
    assert capi.combine_results(parts[::-1]).rot_index == 7


def test_combine_status_rules():
    # a shard that voted nowhere still offers its best rotation (its
    # rotations are candidates of the whole grid); OK if any shard voted
    parts = [res(0.1, 11, capi.DSES_ERR_NO_CANDIDATE), res(0.3, 2)]
    out = capi.combine_results(parts)
    assert out.rot_index == 11 and out.status == capi.DSES_OK
    # no shard voted: NO_CANDIDATE, with the best filled result
    out = capi.combine_results([res(0.4, 5, capi.DSES_ERR_NO_CANDIDATE), res(0.2, 9, capi.DSES_ERR_NO_CANDIDATE)])
    assert out.rot_index == 9 and out.status == capi.DSES_ERR_NO_CANDIDATE
    # shards without rotations are skipped
    empty = res(float("nan"), -1, capi.DSES_ERR_NO_CANDIDATE)
    assert capi.combine_results([empty, res(0.7, 4)]).rot_index == 4
    st, out = capi.dses_combine_results([empty, empty])
    assert st == capi.DSES_ERR_NO_CANDIDATE and out.rot_index == -1 and math.isnan(out.cost)
    # a failed shard cannot be combined
    st, _ = capi.dses_combine_results([res(0.1, 1), res(0.0, 2, capi.DSES_ERR_CUDA)])
    assert st == capi.DSES_ERR_INVALID_ARG


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
    from paper_2502_00115_b300 import capi as c
    from paper_2502_00115_b300 import shard

    c.load()
    # rank k's shard found rotation 100 k + 3 at cost 1 / (k + 1)
    mine = res(1.0 / (rank + 1), 100 * rank + 3, inliers=rank)
    parts = shard.gather_results(mine)
    best = c.combine_results(parts)
    out[rank] = ([p.rot_index for p in parts], best.rot_index, best.inliers, best.cost)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_combine():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        idx, best, inl, cost = out[r]
        assert idx == [3, 103]
        assert best == 103 and inl == 1 and cost == pytest.approx(0.5)
