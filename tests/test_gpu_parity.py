"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small cases compare every rotation; the full-size ModelNet-shaped problem
(294,912 rotations, the benchmark's launch configuration) compares sampled
rotations the oracle can evaluate one by one. See tests/parity.py for the
tolerance rules.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import build, capi, synth
from parity import Report, check_rotations, cost_close, result_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = capi.Context(0)
    yield c
    c.close()


def gpu_params(prob, **over):
    kw = dict(metric=prob.metric, epsilon=prob.epsilon, delta_t=prob.delta_t, tau=prob.tau, huber_h=prob.huber_h,
              t_center=prob.t_center, t_half=prob.t_half, q_milli=prob.q_milli, top_k=prob.top_k,
              refine_top_k=prob.refine_top_k, refine_K=prob.refine_K, refine_delta_r=prob.refine_delta_r)
    kw.update(over)
    return capi.make_params(**kw)


def oracle_params(p, gp, grid_cap):
    """Oracle parameters from the exact FP32 values the GPU received."""
    return oracle.make_params(
        metric=gp.metric, epsilon=float(np.float32(gp.epsilon)),
        delta_t=float(np.float32(gp.delta_t if gp.delta_t > 0 else gp.epsilon)),
        tau=float(np.float32(gp.tau if gp.tau > 0 else 2 * gp.epsilon)),
        huber_h=float(np.float32(gp.huber_h if gp.huber_h > 0 else gp.epsilon)), p=float(np.float32(gp.p)),
        t_center=[float(v) for v in gp.t_center], t_half=[float(v) for v in gp.t_half], q_milli=gp.q_milli,
        top_k=gp.top_k, nn_mode=gp.nn_mode, grid_res=128, grid_cap=float(np.float32(grid_cap)),
        refine_top_k=gp.refine_top_k, refine_K=gp.refine_K, refine_delta_r=gp.refine_delta_r)


# ---------------------------------------------------------------------------
# grids and target preprocessing


@pytest.mark.parametrize("n", [1, 2, 4, 10, 16])
def test_hopf_grid_matches_oracle(ctx, n):
    Rg = ctx.rotation_grid(capi.hopf_grid(n)).astype(np.float64)
    Ro = oracle.hopf_grid(n)
    assert Rg.shape == Ro.shape
    assert np.abs(Rg - Ro).max() <= 1e-6


def test_euler_box_matches_oracle(ctx):
    from scipy.spatial.transform import Rotation

    R0 = Rotation.random(random_state=3).as_matrix()
    Rg = ctx.rotation_grid(capi.euler_box_grid(R0, 3, math.radians(0.3125))).astype(np.float64)
    Ro = oracle.euler_box(R0, 3, math.radians(0.3125))
    assert np.abs(Rg - Ro).max() <= 1e-6


def test_distance_grid_matches_oracle(ctx):
    p = synth.tiny_problem(2)
    cap = 0.08
    t = ctx.create_target(p.Y, grid_cap=cap, grid_res=40)
    D, lo, h, gcap = ctx.distance_grid(t)
    g = oracle.dist_grid(p.Y, 40, float(np.float32(cap)))
    np.testing.assert_allclose(lo, g.lo, rtol=0, atol=1e-6)
    np.testing.assert_allclose(h, g.h, rtol=1e-6)
    assert np.abs(D - g.D).max() <= 2e-6
    assert gcap == np.float32(cap)
    ctx.destroy_target(t)


# ---------------------------------------------------------------------------
# every rotation of the tiny problem


def _run_tiny(ctx, seed, metric, nn_mode, hopf_n=4, **over):
    p = synth.tiny_problem(seed, hopf_n=hopf_n)
    cap = 2 * p.tau
    t = ctx.create_target(p.Y, grid_cap=cap)
    gp = gpu_params(p, metric=metric, nn_mode=nn_mode, **over)
    pb = ctx.problem(t, p.X, capi.hopf_grid(hopf_n), gp)
    P = oracle_params(p, gp, cap)
    n_rot = 72 * hopf_n**3
    if gp.refine_top_k:
        n_rot += gp.refine_top_k * (2 * gp.refine_K + 1) ** 3
    k, V, M, C, r = ctx.debug(pb, n_rot)
    return p, t, pb, P, k, V, M, C, r


@pytest.mark.parametrize("metric,nn", [("trunc_l1", "grid"), ("inlier", "grid"), ("trunc_l2", "brute"),
                                       ("huber", "grid"), ("lp", "brute")])
def test_tiny_every_rotation_matches_oracle(ctx, metric, nn):
    p, t, pb, P, k, V, M, C, r = _run_tiny(ctx, 0, metric, nn, p=0.5)
    grid = oracle.hopf_grid(p.hopf_n)
    ref = oracle.register(p.X, p.Y, grid, P)
    g = oracle.dist_grid(p.Y, 128, P.grid_cap) if nn == "grid" and metric != "inlier" else None
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, range(len(grid)), ref=ref, dist_grid=g)
    print("parity:", rep.summary())  # counted boundary cases, reported with -s
    assert rep.ok(), rep.summary()
    assert rep.vote_exact >= 0.98 * rep.checked, rep.summary()
    assert np.all(np.isfinite(C))  # every rotation is a candidate (q = 0)
    # best rotation: exact, or a near-tie of the oracle's costs
    assert r.status == 0
    if r.rot_index != ref.rot_index:
        assert cost_close(ref.costs[r.rot_index], ref.costs[ref.rot_index], 1), (r.rot_index, ref.rot_index)
    ctx.destroy_target(t)


@pytest.mark.parametrize("over", [dict(q_milli=900), dict(top_k=20), dict(q_milli=500, nn_mode="brute")])
def test_tiny_candidate_filters_match_oracle(ctx, over):
    nn = over.pop("nn_mode", "grid")
    p, t, pb, P, k, V, M, C, r = _run_tiny(ctx, 1, "trunc_l1", nn, **over)
    grid = oracle.hopf_grid(p.hopf_n)
    ref = oracle.register(p.X, p.Y, grid, P)
    g = oracle.dist_grid(p.Y, 128, P.grid_cap) if nn == "grid" else None
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, range(len(grid)), ref=ref, dist_grid=g)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    cand_gpu = set(np.flatnonzero(np.isfinite(C)).tolist())
    cand_ref = set(np.flatnonzero(np.isfinite(ref.costs)).tolist())
    if rep.m_excused == 0 and rep.vote_excused == 0:
        assert cand_gpu == cand_ref
    else:
        assert len(cand_gpu ^ cand_ref) <= rep.m_excused + rep.vote_excused
    if r.rot_index != ref.rot_index:
        assert cost_close(ref.costs[r.rot_index], ref.costs[ref.rot_index], 1)
    ctx.destroy_target(t)


def test_tiny_refinement_pass_matches_oracle(ctx):
    over = dict(refine_top_k=4, refine_K=1, refine_delta_r=math.radians(3.0))
    p, t, pb, P, k, V, M, C, r = _run_tiny(ctx, 2, "trunc_l1", "brute", hopf_n=2, **over)
    grid = oracle.hopf_grid(2)
    ref = oracle.register(p.X, p.Y, grid, P)
    # the oracle's second-pass rotations, rebuilt from its own coarse ranking
    order = sorted(np.flatnonzero(np.isfinite(ref.costs[: len(grid)])), key=lambda i: (ref.costs[i], i))[:4]
    fine = np.concatenate([oracle.euler_box(grid[c], 1, math.radians(3.0)) for c in order])
    allR = np.concatenate([grid, fine])
    rep = check_rotations(p.X, p.Y, allR, P, k, V, M, C, range(len(allR)), ref=ref)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    assert r.rot_index == ref.rot_index or cost_close(ref.costs[r.rot_index], ref.costs[ref.rot_index], 1)
    assert r.cost <= np.nanmin(C[: len(grid)]) + 1e-7
    ctx.destroy_target(t)


def test_histogram_modes_and_launch_shapes_agree(ctx):
    # dense 32-bit, packed 16-bit and slabbed histograms, every points-per-thread
    # variant and fused / separate scoring give identical per-rotation results
    p = synth.modelnet_like_problem(5, m=300, keep=0.7, hopf_n=3)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    gp = gpu_params(p, nn_mode="grid")
    pb = ctx.problem(t, p.X, capi.hopf_grid(3), gp)
    n = 72 * 27
    base = ctx.debug(pb, n)
    variants = [dict(hist_mode=1), dict(hist_mode=2), dict(hist_mode=1, hist_budget_bytes=20000),
                dict(hist_mode=2, hist_budget_bytes=9000), dict(points_per_thread=1), dict(points_per_thread=2),
                dict(points_per_thread=8), dict(fuse_score=0), dict(tile_rotations=1), dict(vote_sparse=2),
                dict(vote_sparse=2, points_per_thread=2), dict(vote_sparse=3), dict(vote_sparse=3, points_per_thread=2),
                dict(vote_sparse=3, hist_mode=1), dict(hist_strides=0), dict(hist_strides=0, hist_mode=1),
                dict(hist_strides=0, vote_sparse=3)]
    defaults = {k: ctx.get_option(k) for k in ("hist_mode", "hist_budget_bytes", "points_per_thread", "fuse_score",
                                               "tile_rotations", "vote_sparse", "hist_strides")}
    try:
        for v in variants:
            for key, val in v.items():
                ctx.set_option(key, val)
            k, V, M, C, r = ctx.debug(pb, n)
            assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2]), v
            np.testing.assert_allclose(C, base[3], rtol=2e-6, err_msg=str(v))
            assert r.rot_index == base[4].rot_index, v
            for key, val in defaults.items():
                ctx.set_option(key, val)
    finally:
        for key, val in defaults.items():
            ctx.set_option(key, val)
    ctx.destroy_target(t)


def test_small_box_lane_private_counters(ctx):
    # a translation box of a few thousand bins (a local search around a prior):
    # the planner's choice against the oracle on sampled rotations, and
    # lane-private counters (hist_mode 3) bit-identical to shared 32-bit
    # counters under every vote path: packed, scalar (1 point per lane),
    # culled and paired culled, odd and padded (even-extent) layouts
    p = synth.modelnet_like_problem(7, hopf_n=2)
    centre = tuple(float(v) for v in np.round(np.asarray(p.t_true) / 0.04) * 0.04)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    # 11^3 bins; then the y range shifted by half a cell: 11 x 10 x 11 (an even extent)
    for first, c in ((True, centre), (False, (centre[0], centre[1] + 0.02, centre[2]))):
        gp = gpu_params(p, nn_mode="grid", t_center=c, t_half=(0.2, 0.2, 0.2))
        pb = ctx.problem(t, p.X, capi.hopf_grid(2), gp)
        n = 72 * 8
        base = ctx.debug(pb, n)
        if first:
            P = oracle_params(p, gp, 2 * p.tau)
            grid = oracle.hopf_grid(2)
            g = oracle.dist_grid(p.Y, 128, P.grid_cap)
            rep = check_rotations(p.X, p.Y, grid, P, base[0], base[1], base[2], base[3], range(0, n, 12),
                                  dist_grid=g)
            print("parity:", rep.summary())
            assert rep.ok(), rep.summary()
        defaults = {k: ctx.get_option(k) for k in ("hist_mode", "points_per_thread", "vote_sparse")}
        try:
            for v in (dict(hist_mode=1), dict(hist_mode=3, points_per_thread=1), dict(hist_mode=3, points_per_thread=8),
                      dict(hist_mode=3, vote_sparse=2), dict(hist_mode=1, vote_sparse=2), dict(hist_mode=3, vote_sparse=3),
                      dict(hist_mode=1, vote_sparse=3, points_per_thread=4), dict(vote_sparse=1),
                      dict(vote_sparse=1, hist_mode=3, points_per_thread=4)):
                for key, val in v.items():
                    ctx.set_option(key, val)
                k, V, M, C, r = ctx.debug(pb, n)
                assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2]), v
                np.testing.assert_allclose(C, base[3], rtol=2e-6, err_msg=str(v))
                for key, val in defaults.items():
                    ctx.set_option(key, val)
        finally:
            for key, val in defaults.items():
                ctx.set_option(key, val)
    ctx.destroy_target(t)


def test_non_cubic_box_every_vote_path(ctx):
    # unequal half-widths (11 x 7 x 15 bins) take the per-axis box test, a
    # cube takes max(|w_x|, |w_y|, |w_z|) < h: each against the oracle on
    # sampled rotations, and every vote path (packed, scalar, culled, paired
    # culled, the dense vote forced, 16- and 32-bit counters) bit-identical
    # to the planner's choice
    p = synth.modelnet_like_problem(11, hopf_n=2)
    centre = tuple(float(v) for v in np.round(np.asarray(p.t_true) / 0.04) * 0.04)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    grid = oracle.hopf_grid(2)
    g = None
    n = 72 * 8
    for half in ((0.2, 0.12, 0.28), (0.16, 0.16, 0.16)):
        gp = gpu_params(p, nn_mode="grid", t_center=centre, t_half=half)
        pb = ctx.problem(t, p.X, capi.hopf_grid(2), gp)
        base = ctx.debug(pb, n)
        P = oracle_params(p, gp, 2 * p.tau)
        g = g if g is not None else oracle.dist_grid(p.Y, 128, P.grid_cap)
        rep = check_rotations(p.X, p.Y, grid, P, base[0], base[1], base[2], base[3], range(0, n, 9), dist_grid=g)
        print("parity:", half, rep.summary())
        assert rep.ok(), rep.summary()
        defaults = {k: ctx.get_option(k) for k in ("hist_mode", "points_per_thread", "vote_sparse")}
        try:
            for v in (dict(points_per_thread=1), dict(points_per_thread=2), dict(points_per_thread=8),
                      dict(hist_mode=1), dict(hist_mode=2), dict(vote_sparse=2), dict(vote_sparse=2, hist_mode=1),
                      dict(vote_sparse=3, points_per_thread=2), dict(vote_sparse=3, hist_mode=1),
                      dict(vote_sparse=1), dict(vote_sparse=1, points_per_thread=2),
                      dict(vote_sparse=1, hist_mode=2, points_per_thread=8)):
                for key, val in v.items():
                    ctx.set_option(key, val)
                k, V, M, C, r = ctx.debug(pb, n)
                assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2]), \
                    (half, v)
                np.testing.assert_allclose(C, base[3], rtol=2e-6, err_msg=str((half, v)))
                for key, val in defaults.items():
                    ctx.set_option(key, val)
        finally:
            for key, val in defaults.items():
                ctx.set_option(key, val)
    ctx.destroy_target(t)


def test_culling_is_conservative_far_from_the_origin(ctx):
    # a target 15,000 lattice units from the origin (the translation box
    # centred there): the staged offsets and thresholds carry FP32 roundings
    # near 1e-3 lattice units, so the culling margin must scale with them;
    # the dense vote, both culled forms and 16-/32-bit counters give
    # bit-identical per-rotation (k*, V, M)
    p = synth.tiny_problem(6, hopf_n=2)
    T = np.array([300.0, -200.0, 100.0])
    Y = (p.Y.astype(np.float64) + T).astype(np.float32)
    t = ctx.create_target(Y, grid_cap=2 * p.tau)
    c = tuple(float(v) for v in np.round((T + np.asarray(p.t_true)) / p.delta_t) * p.delta_t)
    gp = gpu_params(p, nn_mode="grid", t_center=c, t_half=(0.1, 0.1, 0.1))
    pb = ctx.problem(t, p.X, capi.hopf_grid(2), gp)
    n = 72 * 8
    defaults = {k: ctx.get_option(k) for k in ("hist_mode", "points_per_thread", "vote_sparse")}
    try:
        ctx.set_option("vote_sparse", 1)
        base = ctx.debug(pb, n)
        assert base[1].max() > 0
        for v in (dict(vote_sparse=1, points_per_thread=2), dict(vote_sparse=1, hist_mode=2),
                  dict(vote_sparse=2), dict(vote_sparse=3), dict(vote_sparse=2, hist_mode=2),
                  dict(vote_sparse=0)):
            for key, val in v.items():
                ctx.set_option(key, val)
            k, V, M, C, r = ctx.debug(pb, n)
            assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2]), v
            for key, val in defaults.items():
                ctx.set_option(key, val)
    finally:
        for key, val in defaults.items():
            ctx.set_option(key, val)
    ctx.destroy_target(t)


def test_in_box_vote_total(ctx):
    # the sum of every histogram count (last_votes_total) is the number of
    # (rotation, source, target) pairs whose lattice key lies in the box: an
    # FP64 count with the kernel's FP32 rotations (a pair within 1e-5 of a
    # voxel face may go either way), the same under every vote path and
    # counter width
    p = synth.tiny_problem(4, hopf_n=2)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    grid = capi.hopf_grid(2)
    gp = gpu_params(p, nn_mode="grid", t_center=(0.02, -0.04, 0.0), t_half=(0.3, 0.2, 0.24))
    pb = ctx.problem(t, p.X, grid, gp)
    ctx.register(pb)
    total = ctx.get_option("last_votes_total")
    P = oracle_params(p, gp, 2 * p.tau)
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    X, Y = p.X.astype(np.float64), p.Y.astype(np.float64)
    inside = near = 0
    for R in ctx.rotation_grid(grid).astype(np.float64):
        w = (Y[:, None, :] - (X @ R.T)[None, :, :]) / P.delta_t
        k = np.floor(w + 0.5)
        inside += int(np.all((k >= lo) & (k <= hi), axis=-1).sum())
        near += int(np.any(np.abs(w - k + 0.5) * P.delta_t < 1e-5, axis=-1).sum())
        near += int(np.any(np.abs(w - k - 0.5) * P.delta_t < 1e-5, axis=-1).sum())
    assert inside > 0 and abs(total - inside) <= near, (total, inside, near)
    defaults = {k: ctx.get_option(k) for k in ("hist_mode", "points_per_thread", "vote_sparse")}
    try:
        for v in (dict(hist_mode=1), dict(hist_mode=2), dict(points_per_thread=1), dict(points_per_thread=8),
                  dict(vote_sparse=2), dict(vote_sparse=3), dict(vote_sparse=2, hist_mode=2)):
            for key, val in v.items():
                ctx.set_option(key, val)
            ctx.register(pb)
            assert ctx.get_option("last_votes_total") == total, v
            for key, val in defaults.items():
                ctx.set_option(key, val)
    finally:
        for key, val in defaults.items():
            ctx.set_option(key, val)
    ctx.destroy_target(t)


@pytest.mark.parametrize("hist_mode", [0, 1])
def test_even_extent_box_matches_oracle(ctx, hist_mode):
    # a box centred half a cell off the lattice has even extents (90 x 89 x 90
    # here); the vote layout is padded to odd extents and the scan skips the
    # padding: every rotation against the oracle, packed 16-bit and 32-bit slabs
    p = synth.tiny_problem(3)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    gp = gpu_params(p, nn_mode="grid", t_center=(0.01, 0.0, -0.01))
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gp)
    P = oracle_params(p, gp, 2 * p.tau)
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    assert ((hi - lo + 1) % 2 == 0).sum() == 2
    ctx.set_option("hist_mode", hist_mode)
    try:
        k, V, M, C, r = ctx.debug(pb, 72 * p.hopf_n**3)
    finally:
        ctx.set_option("hist_mode", 0)
    grid = oracle.hopf_grid(p.hopf_n)
    ref = oracle.register(p.X, p.Y, grid, P)
    g = oracle.dist_grid(p.Y, 128, P.grid_cap)
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, range(len(grid)), ref=ref, dist_grid=g)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    assert rep.vote_exact >= 0.98 * rep.checked, rep.summary()
    ctx.destroy_target(t)


def test_lane_private_counters_refused_when_they_do_not_fit(ctx):
    p = synth.tiny_problem(2, hopf_n=1)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    pb = ctx.problem(t, p.X, capi.hopf_grid(1), gpu_params(p, nn_mode="grid"))  # 91^3 bins
    ctx.set_option("hist_mode", 3)
    try:
        st, _ = capi.dses_register(ctx.h, pb)
        assert st == capi.DSES_ERR_INVALID_ARG
    finally:
        ctx.set_option("hist_mode", 0)
    ctx.register(pb)  # the context stays usable
    ctx.destroy_target(t)


# ---------------------------------------------------------------------------
# the full-size ModelNet-shaped problem (benchmark configuration), sampled


def test_modelnet_full_size_sampled_rotations(ctx):
    p = synth.modelnet_like_problem(0)
    cap = 2 * p.tau
    t = ctx.create_target(p.Y, grid_cap=cap)
    gp = gpu_params(p, nn_mode="grid")
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gp)
    n = 72 * p.hopf_n**3
    k, V, M, C, r = ctx.debug(pb, n)
    assert r.status == 0 and np.all(np.isfinite(C))
    assert r.rot_index == int(np.lexsort((np.arange(n), C))[0])  # argmin of (cost, index)
    P = oracle_params(p, gp, cap)
    rng = np.random.default_rng(0)
    idx = sorted(set(rng.choice(n, size=40, replace=False).tolist()) | {r.rot_index, int(np.argmax(M))})
    Rs = np.stack([oracle.hopf_rotation(p.hopf_n, i) for i in idx])
    g = oracle.dist_grid(p.Y, 128, P.grid_cap)
    rep = check_rotations(p.X, p.Y, Rs, P, k, V, M, C, idx, dist_grid=g)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    # the winner is a plausible pose (grid resolution ~3.75 degrees)
    ang = np.degrees(np.arccos(np.clip((np.trace(np.array(r.R[:]).reshape(3, 3).T @ p.R_true) - 1) / 2, -1, 1)))
    assert ang < 10.0, ang
    ctx.destroy_target(t)


def test_culled_modes_agree_on_robot_like(ctx):
    # the paired 64-point-group culling (auto here), the 32-point culling and
    # the dense vote give bit-identical per-rotation (k*, V, M), and so do the
    # compact and the bank-spreading histogram strides
    p = synth.robot_like_problem(0, hopf_n=2, refine_top_k=0)
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    pb = ctx.problem(t, p.X, capi.hopf_grid(2), gpu_params(p, nn_mode="grid", huber_h=p.huber_h, refine_top_k=0))
    n = 72 * 8
    base = ctx.debug(pb, n)
    assert ctx.get_option("last_vote_paired") == 1
    try:
        ctx.set_option("hist_strides", 0)
        k, V, M, C, r = ctx.debug(pb, n)
        ctx.set_option("hist_strides", 1)
        assert ctx.get_option("last_vote_paired") == 1
        assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2])
        for mode in (2, 1):
            ctx.set_option("vote_sparse", mode)
            k, V, M, C, r = ctx.debug(pb, n)
            assert ctx.get_option("last_vote_paired") == 0
            assert np.array_equal(k, base[0]) and np.array_equal(V, base[1]) and np.array_equal(M, base[2]), mode
    finally:
        ctx.set_option("vote_sparse", 0)
    ctx.destroy_target(t)


def test_paired_lists_with_16bit_counters_and_many_items(ctx):
    # the paired vote's kept-source lists on the forms the robot-like line
    # does not take: 16-bit counters (a 41^3 box forced to 16 bits, 300
    # sources: one item walks them all, so the lists are used) and two
    # targets per lane (one list per item) on a 40,000-point target (625
    # items per rotation): every rotation's (k*, V, M) bit-identical to the
    # dense vote
    p = synth.robot_like_problem(0, hopf_n=2, refine_top_k=0)
    n = 72 * 8
    defaults = {k: ctx.get_option(k) for k in ("hist_mode", "points_per_thread", "vote_sparse")}
    try:
        t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
        gp = gpu_params(p, nn_mode="grid", refine_top_k=0, t_half=(0.06, 0.06, 0.06))
        pb = ctx.problem(t, p.X[:300], capi.hopf_grid(2), gp)
        ctx.set_option("hist_mode", 2)
        ctx.set_option("vote_sparse", 3)
        paired = ctx.debug(pb, n)
        assert ctx.get_option("last_vote_paired") == 1
        ctx.set_option("vote_sparse", 1)
        dense = ctx.debug(pb, n)
        assert ctx.get_option("last_vote_sparse") == 0
        for a, b in zip(paired[:3], dense[:3]):
            assert np.array_equal(a, b)
        ctx.destroy_target(t)
        for key, val in defaults.items():
            ctx.set_option(key, val)

        big = synth.robot_like_problem(1, m=40000, hopf_n=2, refine_top_k=0)
        t = ctx.create_target(big.Y, grid_cap=big.grid_cap)
        pb = ctx.problem(t, big.X, capi.hopf_grid(2), gpu_params(big, nn_mode="grid", refine_top_k=0))
        ctx.set_option("points_per_thread", 2)
        ctx.set_option("vote_sparse", 3)
        paired = ctx.debug(pb, n)
        assert ctx.get_option("last_vote_paired") == 1
        ctx.set_option("vote_sparse", 1)
        dense = ctx.debug(pb, n)
        for a, b in zip(paired[:3], dense[:3]):
            assert np.array_equal(a, b)
        ctx.destroy_target(t)
    finally:
        for key, val in defaults.items():
            ctx.set_option(key, val)


def test_paired_vote_with_a_few_sources(ctx):
    # 1 to 17 sources on the paired path (forced): a partial tile of the
    # staged offsets is wider than 32 bytes per source, so the staging must be
    # sized by tiles; every rotation's (k*, V, M) bit-identical to the dense vote
    p = synth.robot_like_problem(0, hopf_n=2, refine_top_k=0)
    n = 72 * 8
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    try:
        for ns in (1, 2, 3, 5, 9, 10, 11, 17):
            pb = ctx.problem(t, p.X[:ns], capi.hopf_grid(2), gpu_params(p, nn_mode="grid", refine_top_k=0))
            ctx.set_option("vote_sparse", 3)
            paired = ctx.debug(pb, n)
            assert ctx.get_option("last_vote_paired") == 1
            ctx.set_option("vote_sparse", 1)
            dense = ctx.debug(pb, n)
            assert ctx.get_option("last_vote_sparse") == 0
            for a, b in zip(paired[:3], dense[:3]):
                assert np.array_equal(a, b), ns
    finally:
        ctx.set_option("vote_sparse", 0)
        ctx.destroy_target(t)


# ---------------------------------------------------------------------------
# batching, special cases, invariances


def oracle_ref(p, gp, cap):
    """The oracle's registration of problem p with the GPU's FP32 parameters
    (threaded over rotations: the same arithmetic as its single-threaded path)."""
    import os

    return oracle.register(p.X, p.Y, oracle.hopf_grid(p.hopf_n), oracle_params(p, gp, cap),
                           threads=os.cpu_count() or 1)


def test_batch_equals_solo(ctx):
    probs = [synth.tiny_problem(s, hopf_n=2 + (s % 2)) for s in range(3)]
    probs.append(synth.modelnet_like_problem(9, m=517, keep=0.55, hopf_n=2))
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    pbs = [ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gpu_params(p, nn_mode="grid"))
           for t, p in zip(targets, probs)]
    solo = [capi.result_dict(ctx.register(pb)) for pb in pbs]
    batch = [capi.result_dict(r) for r in ctx.register_batch(pbs)]
    for a, b in zip(solo, batch):
        assert a["rot_index"] == b["rot_index"] and a["inliers"] == b["inliers"] and a["votes"] == b["votes"]
        assert np.array_equal(a["t"], b["t"]) and a["cost"] == b["cost"] and a["status"] == b["status"] == 0
    for p, pb, b in zip(probs, pbs, batch):  # and each against the oracle
        result_matches_oracle(b, oracle_ref(p, pb.params, 2 * p.tau), len(p.X))
    for t in targets:
        ctx.destroy_target(t)


def test_graph_replayed_batches_equal_solo(ctx):
    # call 1 runs the pipeline, call 2 captures it as a CUDA graph and replays,
    # call 3 replays with new source clouds of the same shapes
    probs = [synth.tiny_problem(s, hopf_n=2) for s in range(3)]
    probs.append(synth.modelnet_like_problem(4, m=400, keep=0.6, hopf_n=2))
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    mk = lambda X: [ctx.problem(t, x, capi.hopf_grid(p.hopf_n), gpu_params(p, nn_mode="grid"))
                    for t, p, x in zip(targets, probs, X)]
    X1 = [p.X for p in probs]
    rng = np.random.default_rng(5)
    X2 = [(p.X + rng.normal(scale=0.01, size=p.X.shape)).astype(np.float32) for p in probs]
    import copy

    refs = {}
    for tag, X in (("X1", X1), ("X2", X2)):
        for i, (p, x) in enumerate(zip(probs, X)):
            q = copy.copy(p)
            q.X = x
            refs[(tag, i)] = oracle_ref(q, gpu_params(p, nn_mode="grid"), 2 * p.tau)
    for tag, X in (("X1", X1), ("X1", X1), ("X2", X2), ("X2", X2)):
        pbs = mk(X)
        batch = [capi.result_dict(r) for r in ctx.register_batch(pbs)]
        solo = [capi.result_dict(ctx.register(pb)) for pb in pbs]
        for i, (a, b) in enumerate(zip(solo, batch)):
            assert a["rot_index"] == b["rot_index"] and a["inliers"] == b["inliers"] and a["votes"] == b["votes"]
            assert np.array_equal(a["t"], b["t"]) and a["cost"] == b["cost"]
            result_matches_oracle(b, refs[(tag, i)], len(X[i]))
    for t in targets:
        ctx.destroy_target(t)


def test_destroyed_targets_drop_their_graphs(ctx):
    # captured graphs are keyed by a target id that is never reused: a target
    # created after another was destroyed (its host address may come back)
    # must not replay a graph captured on the old one, and destroying a target
    # frees the graphs that read it
    plain = capi.Context(0)
    plain.set_option("use_graphs", 0)
    base = ctx.get_option("graphs_cached")
    try:
        for s in range(4):
            p = synth.tiny_problem(10 + s, hopf_n=2)
            t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
            gp = gpu_params(p, nn_mode="grid")
            rs = [capi.result_dict(ctx.register(ctx.problem(t, p.X, capi.hopf_grid(2), gp))) for _ in range(3)]
            assert ctx.get_option("graphs_cached") == base + 1
            tp = plain.create_target(p.Y, grid_cap=2 * p.tau)
            ref = capi.result_dict(plain.register(plain.problem(tp, p.X, capi.hopf_grid(2), gp)))
            plain.destroy_target(tp)
            for r in rs:
                assert r["rot_index"] == ref["rot_index"] and r["cost"] == ref["cost"]
                assert np.array_equal(r["t"], ref["t"]) and r["inliers"] == ref["inliers"]
            ctx.destroy_target(t)
            assert ctx.get_option("graphs_cached") == base
    finally:
        plain.close()


def test_autotuned_shapes_give_identical_results(ctx):
    p = synth.modelnet_like_problem(6, m=700, keep=0.7, hopf_n=3)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    pb = ctx.problem(t, p.X, capi.hopf_grid(3), gpu_params(p, nn_mode="grid"))
    ctx.set_option("autotune", 0)  # fixed heuristic shapes
    try:
        base = ctx.debug(pb, 72 * 27)
    finally:
        ctx.set_option("autotune", 1)  # the default: tuned points per thread and rotations per work item
    tuned = ctx.debug(pb, 72 * 27)
    tuned2 = ctx.debug(pb, 72 * 27)
    assert ctx.get_option("last_p_mask") != 0 and ctx.get_option("last_tile_max") >= 1
    forced = []
    for tile in (1, 7, 16):  # rotations per work item forced
        ctx.set_option("tile_rotations", tile)
        try:
            forced.append(ctx.debug(pb, 72 * 27))
            assert ctx.get_option("last_tile_max") == tile
        finally:
            ctx.set_option("tile_rotations", 0)
    for other in [tuned, tuned2] + forced:
        for a, b in zip(base[:3], other[:3]):
            assert np.array_equal(a, b)
        assert other[4].rot_index == base[4].rot_index
    ctx.destroy_target(t)


def test_theorem_case_exact_recovery_on_gpu(ctx):
    rng = np.random.default_rng(8)
    delta = 0.05
    Y = synth.dyadic_cloud(rng, 80, extent=0.8, min_sep_inf=delta)
    grid = oracle.hopf_grid(3)
    r_true = int(rng.integers(len(grid)))
    k_true = np.array([2, -3, 4])
    sub = Y[rng.choice(80, size=30, replace=False)]
    X = (sub - k_true * delta) @ grid[r_true]
    t = ctx.create_target(Y, grid_cap=0.2)
    for metric in ("inlier", "trunc_l1"):
        gp = capi.make_params(metric=metric, epsilon=delta, tau=0.1, t_half=(0.5, 0.5, 0.5))
        r = ctx.register(ctx.problem(t, X, capi.hopf_grid(3), gp))
        assert r.status == 0 and r.rot_index == r_true and r.inliers == 30 and r.votes == 30
        np.testing.assert_allclose(r.t[:], k_true * delta, atol=1e-6)
    ctx.destroy_target(t)


def test_single_source_point_and_ragged_sizes(ctx):
    rng = np.random.default_rng(3)
    for N, M in [(1, 40), (3, 129), (257, 1000), (1500, 2050)]:
        Y = rng.uniform(-0.6, 0.6, size=(M, 3)).astype(np.float32)
        X = rng.uniform(-0.4, 0.4, size=(N, 3)).astype(np.float32)
        t = ctx.create_target(Y, grid_cap=0.1)
        gp = capi.make_params(metric="trunc_l1", epsilon=0.05, tau=0.05, t_half=(0.4, 0.4, 0.4), nn_mode="brute")
        pb = ctx.problem(t, X, capi.hopf_grid(1), gp)
        k, V, Mg, C, r = ctx.debug(pb, 72)
        P = oracle_params(None, gp, 0.1)
        grid = oracle.hopf_grid(1)
        ref = oracle.register(X, Y, grid, P)
        rep = check_rotations(X, Y, grid, P, k, V, Mg, C, range(72), ref=ref)
        assert rep.ok(), (N, M, rep.summary())
        if N == 1:
            assert V.max() == 1
        ctx.destroy_target(t)


def test_no_vote_inside_the_box_reports_no_candidate(ctx):
    Y = np.array([[5.0, 5.0, 5.0], [6.0, 5.0, 5.0], [5.0, 6.0, 5.0]], dtype=np.float32)
    X = np.zeros((4, 3), dtype=np.float32) + np.arange(4, dtype=np.float32)[:, None] * 0.01
    t = ctx.create_target(Y, grid_cap=0.1)
    gp = capi.make_params(metric="trunc_l1", epsilon=0.05, tau=0.05, t_half=(0.2, 0.2, 0.2))
    r = ctx.register(ctx.problem(t, X, capi.hopf_grid(1), gp))
    assert r.status == capi.DSES_ERR_NO_CANDIDATE and r.votes == 0
    ctx.destroy_target(t)


def test_explicit_and_euler_grids_match_oracle(ctx):
    p = synth.tiny_problem(4, hopf_n=2)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    gp = gpu_params(p, nn_mode="brute")
    P = oracle_params(p, gp, 2 * p.tau)
    from scipy.spatial.transform import Rotation

    Rx = Rotation.random(50, random_state=1).as_matrix()
    g, keep = capi.explicit_grid(Rx)
    k, V, M, C, r = ctx.debug(ctx.problem(t, p.X, g, gp), 50)
    ref = oracle.register(p.X, p.Y, Rx.astype(np.float32).astype(np.float64), P)
    rep = check_rotations(p.X, p.Y, Rx.astype(np.float32).astype(np.float64), P, k, V, M, C, range(50), ref=ref)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    eg = capi.euler_box_grid(p.R_true, 2, math.radians(4))
    k, V, M, C, r = ctx.debug(ctx.problem(t, p.X, eg, gp), 125)
    Re = oracle.euler_box(p.R_true, 2, math.radians(4))
    ref = oracle.register(p.X, p.Y, Re, P)
    rep = check_rotations(p.X, p.Y, Re, P, k, V, M, C, range(125), ref=ref)
    print("parity:", rep.summary())
    assert rep.ok(), rep.summary()
    ctx.destroy_target(t)


def test_device_pointers_match_host_pointers(ctx):
    torch = pytest.importorskip("torch")
    p = synth.tiny_problem(6, hopf_n=2)
    Yd = torch.from_numpy(p.Y).cuda()
    Xd = torch.from_numpy(p.X).cuda()
    torch.cuda.synchronize()
    t1 = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    t2 = ctx.create_target_device(Yd.data_ptr(), len(p.Y), grid_cap=2 * p.tau)
    gp = gpu_params(p, nn_mode="grid")
    a = capi.result_dict(ctx.register(ctx.problem(t1, p.X, capi.hopf_grid(2), gp)))
    b = capi.result_dict(ctx.register(ctx.problem(t2, None, capi.hopf_grid(2), gp, src_ptr=Xd.data_ptr(),
                                                  n_src=len(p.X))))
    assert a["rot_index"] == b["rot_index"] and a["cost"] == b["cost"] and np.array_equal(a["t"], b["t"])
    ctx.destroy_target(t1)
    ctx.destroy_target(t2)


def test_translation_equivariance_and_permutation_invariance(ctx):
    rng = np.random.default_rng(12)
    delta = 2.0**-5
    Y = synth.dyadic_cloud(rng, 200, extent=0.7).astype(np.float32)
    X = synth.dyadic_cloud(rng, 60, extent=0.5).astype(np.float32)
    m = np.array([3, -2, 5])
    base = capi.make_params(metric="trunc_l1", epsilon=delta, tau=0.06, t_half=(0.5, 0.5, 0.5), nn_mode="brute")
    shifted = capi.make_params(metric="trunc_l1", epsilon=delta, tau=0.06, t_center=tuple(m * delta),
                               t_half=(0.5, 0.5, 0.5), nn_mode="brute")
    t1 = ctx.create_target(Y, grid_cap=0.2)
    t2 = ctx.create_target((Y + m * delta).astype(np.float32), grid_cap=0.2)
    k1, V1, M1, C1, r1 = ctx.debug(ctx.problem(t1, X, capi.hopf_grid(2), base), 576)
    k2, V2, M2, C2, r2 = ctx.debug(ctx.problem(t2, X, capi.hopf_grid(2), shifted), 576)
    same = np.all(k2 - k1 == m, axis=1) & (V1 == V2)
    assert same.mean() > 0.99
    assert r1.rot_index == r2.rot_index
    perm_x, perm_y = rng.permutation(len(X)), rng.permutation(len(Y))
    t3 = ctx.create_target(Y[perm_y], grid_cap=0.2)
    k3, V3, M3, C3, r3 = ctx.debug(ctx.problem(t3, X[perm_x], capi.hopf_grid(2), base), 576)
    assert np.array_equal(k3, k1) and np.array_equal(V3, V1) and np.array_equal(M3, M1)
    np.testing.assert_allclose(C3, C1, rtol=1e-5)
    assert r3.rot_index == r1.rot_index
    for t in (t1, t2, t3):
        ctx.destroy_target(t)


def test_invalid_arguments_leave_the_context_usable(ctx):
    p = synth.tiny_problem(0, hopf_n=1)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    bad = capi.make_params(metric="trunc_l1", epsilon=-1.0)
    st, _ = capi.dses_register(ctx.h, ctx.problem(t, p.X, capi.hopf_grid(1), bad))
    assert st == capi.DSES_ERR_INVALID_ARG and "epsilon" in capi.dses_last_error(ctx.h)
    st, _ = capi.dses_register(ctx.h, ctx.problem(t, p.X, capi.hopf_grid(0), gpu_params(p)))
    assert st == capi.DSES_ERR_INVALID_ARG
    small_cap = capi.make_params(metric="trunc_l1", epsilon=0.02, tau=1.0)
    st, _ = capi.dses_register(ctx.h, ctx.problem(t, p.X, capi.hopf_grid(1), small_cap))
    assert st == capi.DSES_ERR_INVALID_ARG
    assert capi.dses_set_option(ctx.h, "no_such_option", 1) == capi.DSES_ERR_INVALID_ARG
    # empty clouds are refused, not registered
    st, _ = capi.dses_register(ctx.h, ctx.problem(t, p.X[:0], capi.hopf_grid(1), gpu_params(p)))
    assert st == capi.DSES_ERR_INVALID_ARG
    with pytest.raises(capi.DsesError):
        ctx.create_target(p.Y[:0], grid_cap=2 * p.tau)
    r = ctx.register(ctx.problem(t, p.X, capi.hopf_grid(1), gpu_params(p)))
    assert r.status == 0
    ctx.destroy_target(t)


def test_forced_16bit_counters_refused_when_they_could_overflow(ctx):
    rng = np.random.default_rng(0)
    Y = (rng.normal(scale=0.001, size=(3000, 3))).astype(np.float32)  # every point in one voxel
    X = (rng.normal(scale=0.001, size=(100, 3))).astype(np.float32)
    t = ctx.create_target(Y, grid_cap=0.1)
    ctx.set_option("hist_mode", 2)
    try:
        st, _ = capi.dses_register(ctx.h, ctx.problem(t, X, capi.hopf_grid(1),
                                                      capi.make_params(epsilon=0.05, tau=0.05)))
        assert st == capi.DSES_ERR_INVALID_ARG
    finally:
        ctx.set_option("hist_mode", 0)
    r = ctx.register(ctx.problem(t, X, capi.hopf_grid(1), capi.make_params(epsilon=0.05, tau=0.05)))
    assert r.status == 0 and r.votes > 65535  # 32-bit counters hold it
    ctx.destroy_target(t)


# ---------------------------------------------------------------------------
# serving: results alone and in the mix


def test_serving_staggered_arrivals_with_second_pass_equal_solo(ctx):
    # requests arriving while others run, split over several iterations (two
    # in flight), some with the Euler-box second pass: each result equals the
    # blocking call's
    import time

    probs = [synth.modelnet_like_problem(s, m=400 + 150 * s, hopf_n=3) for s in range(5)]
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    pbs = [ctx.problem(t, p.X, capi.hopf_grid(3),
                       gpu_params(p, nn_mode="grid", refine_top_k=4 if i % 2 else 0, refine_K=1,
                                  refine_delta_r=math.radians(1.0)))
           for i, (t, p) in enumerate(zip(targets, probs))]
    solo = [capi.result_dict(ctx.register(pb)) for pb in pbs]
    ctx.set_option("serve_iter_pairs", 20_000_000)
    try:
        tickets = [ctx.submit(pb) for pb in pbs[:2]]
        time.sleep(0.01)
        tickets += [ctx.submit(pb) for pb in pbs[2:]]
        out = {}
        deadline = time.time() + 120
        while len(out) < len(tickets) and time.time() < deadline:
            for tk in tickets:
                if tk not in out:
                    st, r = ctx.poll(tk)
                    if st != capi.DSES_NOT_READY:
                        assert st == capi.DSES_OK
                        out[tk] = capi.result_dict(r)
            time.sleep(0.002)
        assert len(out) == len(tickets)
    finally:
        ctx.set_option("serve_iter_pairs", 150_000_000_000)
    for tk, a, p, pb in zip(tickets, solo, probs, pbs):
        b = out[tk]
        assert a["rot_index"] == b["rot_index"] and a["inliers"] == b["inliers"] and a["votes"] == b["votes"]
        assert np.array_equal(a["t"], b["t"]) and a["cost"] == b["cost"]
        result_matches_oracle(b, oracle_ref(p, pb.params, 2 * p.tau), len(p.X))
    for t in targets:
        ctx.destroy_target(t)


def test_serving_results_equal_solo(ctx):
    import time

    probs = [synth.tiny_problem(s, hopf_n=2 + (s % 3)) for s in range(6)]
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    pbs = [ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gpu_params(p, nn_mode="grid"))
           for t, p in zip(targets, probs)]
    solo = [capi.result_dict(ctx.register(pb)) for pb in pbs]
    ctx.set_option("serve_tile_rotations", 300)
    try:
        tickets = [ctx.submit(pb) for pb in pbs]
        out = {}
        deadline = time.time() + 60
        while len(out) < len(tickets) and time.time() < deadline:
            for tk in tickets:
                if tk in out:
                    continue
                st, r = ctx.poll(tk)
                if st != capi.DSES_NOT_READY:
                    assert st == capi.DSES_OK
                    out[tk] = capi.result_dict(r)
            time.sleep(0.002)
        assert len(out) == len(tickets)
        assert capi.dses_poll(ctx.h, tickets[0])[0] == capi.DSES_ERR_UNKNOWN_TICKET
    finally:
        ctx.set_option("serve_tile_rotations", 1 << 30)
    for tk, a, p, pb in zip(tickets, solo, probs, pbs):
        b = out[tk]
        assert a["rot_index"] == b["rot_index"] and a["inliers"] == b["inliers"] and a["votes"] == b["votes"]
        assert np.array_equal(a["t"], b["t"]) and a["cost"] == b["cost"]
        result_matches_oracle(b, oracle_ref(p, pb.params, 2 * p.tau), len(p.X))
    for t in targets:
        ctx.destroy_target(t)
