"""Parity of the CUDA Algorithm 1 validator (dses_exhaustive_search) with the
FP64 oracle's exhaustive search: every (rotation, lattice translation) error,
the argmin, and agreement with Algorithm 2 where the paper's Theorem fixes it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import build, capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = capi.Context(0)
    yield c
    c.close()


def small_problem(seed):
    p = synth.tiny_problem(seed)
    rng = np.random.default_rng(seed + 100)
    X = p.X[rng.choice(len(p.X), 48, replace=False)]
    centre = tuple(float(v) for v in np.round(np.asarray(p.t_true) / 0.02) * 0.02)
    return p, X, centre


def params(metric, centre, half=0.06):
    return dict(metric=metric, epsilon=0.02, tau=0.04, huber_h=0.02, p=0.5, t_center=centre,
                t_half=(half, half, half))


@pytest.mark.parametrize("metric", ["trunc_l1", "trunc_l2", "huber", "lp", "inlier"])
def test_every_entry_matches_oracle(ctx, metric):
    p, X, centre = small_problem(1)
    rots = oracle.euler_box(p.R_true, 1, math.radians(4.0))
    grid = capi.euler_box_grid(p.R_true, 1, math.radians(4.0))
    kw = params(metric, centre)
    tgt = ctx.create_target(p.Y, grid_cap=0.1)
    pb = ctx.problem(tgt, X, grid, capi.make_params(**kw))
    Rg = ctx.rotation_grid(grid).astype(np.float64)  # the FP32 rotations the kernel used
    P = oracle.make_params(**{k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in kw.items()})
    P.t_center[:] = [float(np.float32(v)) for v in centre]
    P.t_half[:] = [float(np.float32(kw["t_half"][0]))] * 3
    cost_o, cnt_o, best_o, _ = oracle.exhaustive(X, p.Y, Rg, P)
    n = cost_o.size
    r, cost_g = ctx.exhaustive(pb, n)
    cost_g = cost_g.reshape(cost_o.shape).astype(np.float64)
    if metric == "inlier":
        # a count may flip only through a point within 1e-5 of epsilon
        bad = np.argwhere(cost_g != cost_o)
        assert len(bad) <= 0.01 * n
        lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
        E = hi - lo + 1
        for rr, ti in bad:
            k = np.array([ti // (E[1] * E[2]), (ti // E[2]) % E[1], ti % E[2]]) + lo
            _, nb = oracle.inliers(X, p.Y, Rg[rr], k * P.delta_t, P.epsilon)
            assert abs(cost_g[rr, ti] - cost_o[rr, ti]) <= nb
    else:
        np.testing.assert_allclose(cost_g, cost_o, rtol=1e-4, atol=1e-6 * len(X))
    flat = cost_o.reshape(-1)
    gi = r.rot_index * cost_o.shape[1]
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    E = hi - lo + 1
    k = np.rint(np.array(r.t[:], np.float64) / P.delta_t).astype(int) - lo
    gi += (k[0] * E[1] + k[1]) * E[2] + k[2]
    assert gi == best_o or flat[gi] <= flat[best_o] + 1e-4 * max(1.0, abs(flat[best_o])) + (metric == "inlier")
    ctx.destroy_target(tgt)


def test_planted_pose_is_found_exactly(ctx):
    rng = np.random.default_rng(5)
    delta = 0.05
    Y = synth.dyadic_cloud(rng, 300, extent=0.5, min_sep_inf=delta).astype(np.float32)
    grid = capi.hopf_grid(1)
    Rg = ctx.rotation_grid(grid).astype(np.float64)
    r_true, k_true = 41, np.array([2, -1, 1])
    X = ((Y[:60].astype(np.float64) - k_true * delta) @ Rg[r_true]).astype(np.float32)
    tgt = ctx.create_target(Y, grid_cap=0.2)
    pb = ctx.problem(tgt, X, grid, capi.make_params(metric="trunc_l1", epsilon=delta, tau=0.1,
                                                    t_half=(0.15, 0.15, 0.15)))
    r, _ = ctx.exhaustive(pb)
    assert r.rot_index == r_true
    np.testing.assert_allclose(np.array(r.t[:]), k_true * delta, atol=1e-6)
    assert r.inliers == 60 and r.cost < 1e-3
    # Algorithm 2 on the same problem reaches the same pose (the Theorem's case)
    rr = ctx.register(pb)
    assert rr.rot_index == r_true and rr.inliers == 60
    ctx.destroy_target(tgt)


def test_dses_cost_is_never_below_the_exhaustive_optimum(ctx):
    p, X, centre = small_problem(3)
    grid = capi.euler_box_grid(p.R_true, 1, math.radians(5.0))
    kw = params("trunc_l2", centre)
    tgt = ctx.create_target(p.Y, grid_cap=0.1)
    pb = ctx.problem(tgt, X, grid, capi.make_params(nn_mode="brute", **kw))
    ex, _ = ctx.exhaustive(pb)
    ds = ctx.register(pb)
    assert ds.cost >= ex.cost * (1 - 1e-5) - 1e-7
    ctx.destroy_target(tgt)


def test_exhaustive_limits_are_enforced(ctx):
    rng = np.random.default_rng(0)
    big = rng.uniform(-1, 1, (12289, 3)).astype(np.float32)
    tgt = ctx.create_target(big, grid_cap=0.1)
    pb = ctx.problem(tgt, big[:10], capi.hopf_grid(1), capi.make_params(epsilon=0.05, t_half=(0.1, 0.1, 0.1)))
    st, _, _ = capi.dses_exhaustive_search(ctx.h, pb)
    assert st == capi.DSES_ERR_INVALID_ARG
    ctx.destroy_target(tgt)
    small = big[:500]
    tgt = ctx.create_target(small, grid_cap=0.1)
    pb = ctx.problem(tgt, small[:10], capi.hopf_grid(1), capi.make_params(epsilon=0.05, t_half=(0.1, 0.1, 0.1)))
    st, _, _ = capi.dses_exhaustive_search(ctx.h, pb, 10)  # capacity below 72 x 125
    assert st == capi.DSES_ERR_INVALID_ARG
    r, cost = ctx.exhaustive(pb, 72 * 125)
    assert cost.shape == (72 * 125,) and np.isfinite(cost).all()
    assert abs(cost.min() - r.cost) <= 1e-6 * max(1.0, r.cost)
    ctx.destroy_target(tgt)
