"""Rotation-sharded registration across processes, one GPU each.

Algorithm 2 scores every rotation of the grid on its own, so one
registration splits into contiguous rotation ranges: every rank registers its
range on its own GPU (dses_register_shard), the ranks all-gather their
results as raw dses_result structs through torch.distributed, and every rank
combines them (dses_combine_results: the lexicographic minimum of (cost,
rotation index), the order of the kernels' argmin). The only exchange is one
result struct per rank; no data-path collective runs.
"""
import ctypes

import torch
import torch.distributed as dist

from . import capi


def gather_results(r: capi.dses_result, group=None) -> list:
    """Every rank's dses_result, in rank order (an all-gather of the raw
    structs: CPU tensors under gloo, CUDA tensors of the current device under
    NCCL)."""
    raw = ctypes.string_at(ctypes.addressof(r), ctypes.sizeof(r))
    t = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    return [capi.dses_result.from_buffer_copy(p.cpu().numpy().tobytes()) for p in parts]


def register_sharded(ctx: capi.Context, pb: capi.dses_problem, group=None) -> capi.dses_result:
    """The registration of pb with its grid split over the group's ranks; every
    rank returns the same result, equal to ctx.register(pb) on one GPU
    (pb's q_milli, top_k and refine_top_k must be 0)."""
    mine = ctx.register_shard(pb, dist.get_rank(group), dist.get_world_size(group))
    return capi.combine_results(gather_results(mine, group))
