"""Rotation-sharded registration across processes, one GPU each.

Algorithm 2 treats every rotation of the grid on its own, so one
registration splits into contiguous rotation ranges, one per rank, each
registered on the rank's own GPU. The ranks meet only where Algorithm 2
reduces over all rotations (the best inlier count M* of the q filter, the
top-k keys, the second pass's centres and the final argmin); the library
makes those exchanges through an all-gather callback, which this module
implements over torch.distributed (CPU tensors under gloo, CUDA tensors of
the current device under NCCL). No data-path collective runs: each exchange
is a few bytes per rank.
"""
import ctypes

import torch
import torch.distributed as dist

from . import capi


def allgather_bytes(mine: bytes, group=None) -> list:
    """Every rank's bytes (all of the same length), in rank order."""
    t = torch.frombuffer(bytearray(mine), dtype=torch.uint8)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    return [p.cpu().numpy().tobytes() for p in parts]


def gather_results(r: capi.dses_result, group=None) -> list:
    """Every rank's dses_result, in rank order (an all-gather of the raw structs)."""
    raw = ctypes.string_at(ctypes.addressof(r), ctypes.sizeof(r))
    return [capi.dses_result.from_buffer_copy(p) for p in allgather_bytes(raw, group)]


def allgather_callback(group=None):
    """The library's all-gather callback over the group (keep it alive for the call)."""
    return capi.make_allgather(lambda mine: allgather_bytes(mine, group))


def register_sharded(ctx: capi.Context, pb: capi.dses_problem, group=None) -> capi.dses_result:
    """The registration of pb with its grid (and second pass) split over the
    group's ranks; every rank returns the same result, equal to ctx.register(pb)
    on one GPU, for any q_milli, top_k and refine_top_k."""
    cb = allgather_callback(group)
    return ctx.register_sharded(pb, dist.get_rank(group), dist.get_world_size(group), cb)


def register_shard_only(ctx: capi.Context, pb: capi.dses_problem, group=None) -> capi.dses_result:
    """The same with no exchange but the final one (dses_register_shard, then an
    all-gather of the results and dses_combine_results): every rotation must be
    a candidate (q_milli = top_k = refine_top_k = 0)."""
    mine = ctx.register_shard(pb, dist.get_rank(group), dist.get_world_size(group))
    return capi.combine_results(gather_results(mine, group))
