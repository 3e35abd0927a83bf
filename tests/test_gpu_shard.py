"""Rotation sharding on one GPU: the shards of a registration, run one after
another in one context, recombine (dses_combine_results) to exactly the
result of the whole registration, on every vote path and grid kind."""
import math

import numpy as np
import pytest

from paper_2502_00115_b300 import build, capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = capi.Context(0)
    yield c
    c.close()


def same(a: capi.dses_result, b: capi.dses_result):
    assert a.rot_index == b.rot_index
    assert np.float32(a.cost).tobytes() == np.float32(b.cost).tobytes()
    assert (a.inliers, a.votes, a.status) == (b.inliers, b.votes, b.status)
    assert list(a.R) == list(b.R) and list(a.t) == list(b.t)


def run_shards(ctx, pb, n_rot, world):
    parts = []
    for k in range(world):
        r = ctx.register_shard(pb, k, world)
        b, e = capi.shard_range(n_rot, k, world)
        assert (b <= r.rot_index < e) if e > b else r.rot_index == -1
        parts.append(r)
    return capi.combine_results(parts[::-1])


@pytest.mark.parametrize("world", [1, 3, 8])
def test_modelnet_shards_recombine(ctx, world):
    p = synth.modelnet_like_problem(2, hopf_n=4)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, tau=p.tau, t_half=p.t_half)
    pb = ctx.problem(t, p.X, capi.hopf_grid(4), pr)
    same(run_shards(ctx, pb, 72 * 64, world), ctx.register(pb))
    ctx.destroy_target(t)


def test_culled_robot_like_shards_recombine(ctx):
    p = synth.robot_like_problem(0, hopf_n=2, refine_top_k=0)
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, tau=p.tau, huber_h=p.huber_h, t_half=p.t_half)
    pb = ctx.problem(t, p.X, capi.hopf_grid(2), pr)
    whole = ctx.register(pb)
    assert ctx.get_option("last_vote_sparse") == 1
    same(run_shards(ctx, pb, 72 * 8, 4), whole)
    ctx.destroy_target(t)


def test_euler_box_and_explicit_grids_and_empty_shards(ctx):
    p = synth.tiny_problem(3)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    pr = capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau, t_half=(0.5, 0.5, 0.5))
    box = capi.euler_box_grid(p.R_true, 3, math.radians(4.0))
    pb = ctx.problem(t, p.X, box, pr)
    same(run_shards(ctx, pb, 343, 5), ctx.register(pb))
    R = ctx.rotation_grid(capi.hopf_grid(1))
    g, keep = capi.explicit_grid(R)
    pb = ctx.problem(t, p.X, g, pr)
    whole = ctx.register(pb)
    same(run_shards(ctx, pb, len(R), 2), whole)
    same(run_shards(ctx, pb, len(R), 100), whole)  # 28 shards without rotations
    ctx.destroy_target(t)


def test_shards_refuse_filters_and_second_passes(ctx):
    p = synth.tiny_problem(0)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    for over in (dict(q_milli=900), dict(top_k=10), dict(refine_top_k=2, refine_K=1, refine_delta_r=0.05)):
        pr = capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau, **over)
        pb = ctx.problem(t, p.X, capi.hopf_grid(1), pr)
        st, _ = capi.dses_register_shard(ctx.h, pb, 0, 2)
        assert st == capi.DSES_ERR_INVALID_ARG, over
    pr = capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau)
    pb = ctx.problem(t, p.X, capi.hopf_grid(1), pr)
    for k, w in ((2, 2), (-1, 2), (0, 0)):
        st, _ = capi.dses_register_shard(ctx.h, pb, k, w)
        assert st == capi.DSES_ERR_INVALID_ARG
    ctx.register(pb)  # the context stays usable
    ctx.destroy_target(t)
