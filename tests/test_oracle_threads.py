"""The oracle's threaded entry points against its single-threaded path, which
the pins check (no GPU). The threaded paths time the CPU baseline and compute
the oracle values of the larger parity cases (the stored ModelNet-shaped
values, the batch and serving checks, the robot-like distance grid); they fan
rotations or grid planes over host threads with the same arithmetic, so
every output must be identical bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import synth


@pytest.fixture(scope="module")
def tiny():
    p = synth.tiny_problem(1, hopf_n=2)
    return p, oracle.hopf_grid(2)


def _same_result(a, b):
    return (a.status, a.rot_index, a.votes, a.inliers) == (b.status, b.rot_index, b.votes, b.inliers) and \
        a.cost == b.cost and np.array_equal(a.R, b.R) and np.array_equal(a.t, b.t)


@pytest.mark.parametrize("kw", [
    dict(nn_mode="brute"),
    dict(nn_mode="brute", metric="huber", q_milli=900),
    dict(nn_mode="brute", metric="inlier", top_k=20),
    dict(nn_mode="brute", metric="trunc_l2", refine_top_k=2, refine_K=1, refine_delta_r=0.02),
    dict(nn_mode="grid", grid_res=32),
])
def test_threaded_registration_equals_single_threaded(tiny, kw):
    p, grid = tiny
    P = oracle.params_from_problem(p, **kw)
    a = oracle.register(p.X, p.Y, grid, P)
    b = oracle.register(p.X, p.Y, grid, P, threads=4)
    for f in ("k", "V", "M", "n_boundary_pairs", "n_boundary_points"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    # rotations a filter leaves unscored carry NaN on both paths
    assert np.array_equal(a.costs, b.costs, equal_nan=True)
    assert _same_result(a, b)
    assert _same_result(a, oracle.register_threads(p.X, p.Y, grid, P, 3))


def test_threaded_and_prebuilt_distance_fields_equal_single_threaded(tiny):
    p, grid = tiny
    P = oracle.params_from_problem(p, nn_mode="grid", grid_res=32)
    g1 = oracle.dist_grid(p.Y, 32, P.grid_cap)
    g4 = oracle.dist_grid(p.Y, 32, P.grid_cap, threads=4)
    assert np.array_equal(g1.D, g4.D) and np.array_equal(g1.lo, g4.lo) and np.array_equal(g1.h, g4.h)
    a = oracle.register(p.X, p.Y, grid, P)
    for th in (1, 4):
        field = oracle.Field(p.Y, 32, P.grid_cap, threads=th)
        try:
            assert _same_result(a, oracle.register_field_threads(p.X, p.Y, grid, P, field, 3)), th
        finally:
            field.close()


def test_single_rotation_evaluation_equals_registration(tiny):
    p, grid = tiny
    P = oracle.params_from_problem(p, nn_mode="brute")
    a = oracle.register(p.X, p.Y, grid, P)
    for r in sorted({0, 17, 300, len(grid) - 1, a.rot_index, int(np.argmax(a.V))}):
        k, V, M, nbp, nbm = oracle.eval_rotation(p.X, p.Y, grid[r], P)
        assert np.array_equal(k, a.k[r]) and V == a.V[r] and M == a.M[r], r
        assert nbp == a.n_boundary_pairs[r] and nbm == a.n_boundary_points[r], r
