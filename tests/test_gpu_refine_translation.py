"""Parity of the CUDA sub-voxel translation refinement (dses_refine_translation)
with the FP64 oracle: the mean of y_nn(i) - R x_i over the inlier pairs at a
pose, iterated. Inlier membership and the nearest target may differ only for
points the oracle flags (distance within 1e-5 of epsilon, or a second-nearest
target within 1e-5 of the nearest); where it flags none the counts must be
equal and the translations agree to 1e-5.
"""
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


def oracle_steps(X, Y, R, t, eps, iterations):
    t = np.asarray(t, np.float64)
    flagged = 0
    n = 0
    for _ in range(iterations):
        # the GPU adds t to R x in FP32; the oracle takes the same FP32 value of t
        t32 = t.astype(np.float32).astype(np.float64)
        t, n, nb, nt = oracle.refine_translation(X, Y, R, t32, eps)
        flagged += nb + nt
    return t, n, flagged


def check(ctx, target, X, Y, R, t, eps, iterations):
    R32 = np.asarray(R, np.float32)
    tg, ng = ctx.refine_translation(target, X, R32, np.asarray(t, np.float32), eps, iterations)
    to, no, flagged = oracle_steps(X, Y, R32.astype(np.float64), t, float(np.float32(eps)), iterations)
    if flagged == 0:
        assert ng == no
        np.testing.assert_allclose(tg, to, atol=1e-5, rtol=0)
    else:  # a flagged point may flip; its effect on the mean is bounded by eps / n
        assert abs(ng - no) <= flagged
        assert np.abs(tg - to).max() <= 1e-5 + 2 * eps * flagged / max(no, 1)
    return tg, ng, to, no


@pytest.mark.parametrize("iterations", [1, 3])
def test_refinement_at_the_registered_pose_matches_oracle(ctx, iterations):
    p = synth.modelnet_like_problem(1, hopf_n=4)
    tgt = ctx.create_target(p.Y, grid_cap=0.1)
    pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, tau=p.tau, t_half=p.t_half)
    r = capi.result_dict(ctx.register(ctx.problem(tgt, p.X, capi.hopf_grid(4), pr)))
    tg, ng, to, no = check(ctx, tgt, p.X, p.Y, r["R"], r["t"], p.epsilon, iterations)
    assert ng > 0
    ctx.destroy_target(tgt)


@pytest.mark.parametrize("n_src", [1, 255, 257, 4099])
def test_ragged_source_sizes_match_oracle(ctx, n_src):
    rng = np.random.default_rng(n_src)
    Y = rng.uniform(-0.5, 0.5, (3000, 3)).astype(np.float32)
    R = np.eye(3)
    t = np.array([0.01, -0.02, 0.015])
    X = (Y[rng.choice(3000, n_src, replace=n_src > 3000)] - t + rng.normal(0, 0.002, (n_src, 3))).astype(np.float32)
    tgt = ctx.create_target(Y, grid_cap=0.1)
    check(ctx, tgt, X, Y, R, t + 0.004, 0.03, 2)
    ctx.destroy_target(tgt)


def test_large_target_sampled_against_oracle(ctx):
    # robot-sized clouds: 5,000 source points against a 20,000-point target
    p = synth.robot_like_problem(0)
    tgt = ctx.create_target(p.Y, grid_cap=0.02)
    start = np.asarray(p.t_true, np.float64) + np.array([0.0012, -0.0009, 0.0011])
    check(ctx, tgt, p.X, p.Y, np.asarray(p.R_true, np.float32), start, p.epsilon, 1)
    ctx.destroy_target(tgt)


def test_no_inlier_keeps_translation_and_device_source_matches_host(ctx):
    import torch

    rng = np.random.default_rng(9)
    Y = rng.uniform(-1, 1, (500, 3)).astype(np.float32)
    X = Y[:200] + np.float32(0.003)
    tgt = ctx.create_target(Y, grid_cap=0.1)
    far = np.array([40.0, 0.0, 0.0], np.float32)
    tr, n = ctx.refine_translation(tgt, X, np.eye(3), far, 0.02)
    assert n == 0
    np.testing.assert_array_equal(tr, far)
    th, nh = ctx.refine_translation(tgt, X, np.eye(3), np.zeros(3), 0.02, 2)
    Xd = torch.from_numpy(X).cuda()
    torch.cuda.synchronize()
    st, td, nd = capi.dses_refine_translation(ctx.h, tgt, Xd.data_ptr(), len(X), 1, np.eye(3), np.zeros(3), 0.02, 2)
    assert st == capi.DSES_OK
    assert nd == nh
    np.testing.assert_array_equal(td, th)
    ctx.destroy_target(tgt)


def test_invalid_refinement_arguments(ctx):
    Y = np.random.default_rng(1).uniform(-1, 1, (100, 3)).astype(np.float32)
    tgt = ctx.create_target(Y, grid_cap=0.1)
    X = Y[:10]
    bad = [
        dict(epsilon=0.0), dict(epsilon=float("nan")), dict(iterations=0), dict(iterations=65),
        dict(t=np.array([np.inf, 0, 0], np.float32)),
    ]
    for b in bad:
        kw = dict(R=np.eye(3), t=np.zeros(3), epsilon=0.02, iterations=1)
        kw.update(b)
        st, _, _ = capi.dses_refine_translation(ctx.h, tgt, X, len(X), 0, kw["R"], kw["t"], kw["epsilon"],
                                                kw["iterations"])
        assert st == capi.DSES_ERR_INVALID_ARG, b
    st, _, _ = capi.dses_refine_translation(ctx.h, tgt, X, 0, 0, np.eye(3), np.zeros(3), 0.02, 1)
    assert st == capi.DSES_ERR_INVALID_ARG
    tr, n = ctx.refine_translation(tgt, X, np.eye(3), np.zeros(3), 0.02)  # still usable
    assert n == 10
    ctx.destroy_target(tgt)
