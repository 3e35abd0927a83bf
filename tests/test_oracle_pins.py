"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published table (HEALPix base
pixels), a library routine (scipy's Euler rotations, cKDTree nearest
neighbours, RegularGridInterpolator), brute force over every lattice cell with
an independent voxel-membership test, or a special case of the paper's
Theorem (Section IV-B) and Lemma 1 (Eq. 5) whose answer is known by
construction.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle
from paper_2502_00115_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# rotation grid


def test_healpix_base_pixels_match_published_layout():
    rows = np.loadtxt(os.path.join(GOLDEN, "healpix_nside1.txt"))
    th, ph = oracle.healpix_centres(1)
    np.testing.assert_allclose(np.cos(th), rows[:, 1], atol=1e-12)
    np.testing.assert_allclose(ph / np.pi, rows[:, 2], atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 10, 16])
def test_healpix_rings_are_equal_area_quadrature(n):
    # Equal-area pixels integrate low-order moments of the uniform sphere
    # measure: E[z] = E[x] = E[y] = 0, E[z^2] = 1/3 up to O(1/n^2).
    th, ph = oracle.healpix_centres(n)
    assert len(th) == 12 * n * n
    z = np.cos(th)
    x, y = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph)
    assert abs(z.mean()) < 1e-12 and abs(x.mean()) < 1e-12 and abs(y.mean()) < 1e-12
    assert abs((z * z).mean() - 1 / 3) < 0.06 / n**2
    # 4n - 1 rings, ring sizes 4i in the caps and 4n on the belt
    _, counts = np.unique(np.round(z, 12), return_counts=True)
    expect = sorted([4 * i for i in range(1, n)] * 2 + [4 * n] * (2 * n + 1))
    assert sorted(counts.tolist()) == expect


@pytest.mark.parametrize("n", [1, 2, 4])
def test_hopf_grid_is_rotations_with_fiber_structure(n):
    R = oracle.hopf_grid(n)
    assert R.shape == (72 * n**3, 3, 3)
    I = np.einsum("rij,rkj->rik", R, R)
    np.testing.assert_allclose(I, np.broadcast_to(np.eye(3), I.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    th, ph = oracle.healpix_centres(n)
    per = 6 * n
    # Hopf fibration: every rotation of one fiber sends e_x (through R^T) to the
    # fiber's base point on S^2, and neighbouring fiber samples differ by a
    # rotation about x of 2 pi / (6n).
    base = np.stack([np.cos(th), -np.sin(th) * np.sin(ph), np.sin(th) * np.cos(ph)], axis=1)
    np.testing.assert_allclose(R[:, 0, :], np.repeat(base, per, axis=0), atol=1e-12)
    step = Rotation.from_rotvec([2 * np.pi / per, 0, 0]).as_matrix()
    for p in range(0, 12 * n * n, max(1, n)):
        for k in range(per - 1):
            A = R[p * per + k + 1] @ R[p * per + k].T
            np.testing.assert_allclose(A, step, atol=1e-12)


def test_hopf_grid_distinct_and_covering():
    cover = {}
    rng = np.random.default_rng(1)
    probe = Rotation.random(3000, random_state=rng).as_quat()  # (x, y, z, w)
    for n in (1, 2, 4):
        q = Rotation.from_matrix(oracle.hopf_grid(n)).as_quat()
        if n <= 2:
            G = np.abs(q @ q.T)
            np.fill_diagonal(G, 0)
            assert G.max() < 1 - 1e-9  # no duplicates up to sign
        d = np.abs(probe @ q.T).max(axis=1)
        cover[n] = np.degrees(2 * np.arccos(np.clip(d.min(), -1, 1)))
    assert cover[4] < 20.0
    assert 1.4 < cover[1] / cover[2] < 2.8 and 1.4 < cover[2] / cover[4] < 2.8


def test_hopf_rotation_matches_grid():
    R = oracle.hopf_grid(3)
    for r in (0, 1, 17, 500, len(R) - 1):
        np.testing.assert_array_equal(oracle.hopf_rotation(3, r), R[r])


def test_euler_box_matches_scipy_intrinsic_zyx():
    rng = np.random.default_rng(3)
    R0 = Rotation.random(random_state=rng).as_matrix()
    K, dr = 2, math.radians(1.7)
    box = oracle.euler_box(R0, K, dr)
    w = 2 * K + 1
    for a, b, c in itertools.product(range(w), repeat=3):
        ang = [(a - K) * dr, (b - K) * dr, (c - K) * dr]
        ref = R0 @ Rotation.from_euler("ZYX", ang).as_matrix()
        np.testing.assert_allclose(box[(a * w + b) * w + c], ref, atol=1e-14)


def test_lattice_box_closed_form():
    lo, hi = oracle.lattice_box((0, 0, 0), (0.9, 0.9, 0.9), 0.02)
    assert lo.tolist() == [-45] * 3 and hi.tolist() == [45] * 3
    lo, hi = oracle.lattice_box((0.1, -0.1, 0.0), (0.05, 0.05, 0.04), 0.04)
    assert lo.tolist() == [2, -3, -1] and hi.tolist() == [3, -2, 1]


# ---------------------------------------------------------------------------
# vote: Lemma 1 / Eq. 5 on the delta_t lattice


def _brute_mode(X, Y, R, delta, lo, hi):
    """Mode by enumerating every lattice cell: a pair supports cell k iff
    y_j - R x_i lies in the half-open voxel [k - 1/2, k + 1/2) delta."""
    T = (Y[None, :, :] - (X @ R.T)[:, None, :]).reshape(-1, 3)
    best, bestk = 0, tuple(lo)
    for k in itertools.product(*[range(l, h + 1) for l, h in zip(lo, hi)]):
        c = np.asarray(k) * delta
        inside = np.all((T >= c - delta / 2) & (T < c + delta / 2), axis=1)
        cnt = int(inside.sum())
        if cnt > best:  # lexicographic enumeration: ties keep the first
            best, bestk = cnt, k
    return np.asarray(bestk), best


@pytest.mark.parametrize("seed", range(6))
def test_vote_mode_equals_brute_force_over_lattice(seed):
    rng = np.random.default_rng(seed)
    delta = 0.125
    N, M = 5, 9
    X = rng.uniform(-0.4, 0.4, size=(N, 3))
    R = Rotation.random(random_state=rng).as_matrix()
    t = rng.uniform(-0.3, 0.3, size=3)
    Y = np.concatenate([(X[:3] @ R.T) + t + rng.normal(scale=0.01, size=(3, 3)),
                        rng.uniform(-0.6, 0.6, size=(M - 3, 3))])
    lo, hi = oracle.lattice_box((0.05, -0.05, 0), (0.5, 0.5, 0.45), delta)
    k, V, nb = oracle.vote(X, Y, R, delta, lo, hi)
    assert nb == 0
    kb, Vb = _brute_mode(X, Y, R, delta, lo, hi)
    assert V == Vb and k.tolist() == kb.tolist()
    assert V >= 2  # the planted translates agree


def test_vote_single_source_point_closed_form():
    # N = 1 and targets pairwise >= delta apart in the inf-norm: every in-box key
    # is distinct, so V = 1 and the mode is the lexicographically smallest key.
    rng = np.random.default_rng(7)
    delta = 0.05
    Y = synth.dyadic_cloud(rng, 40, extent=0.5, min_sep_inf=delta)
    X = np.array([[0.013, -0.021, 0.007]])
    R = Rotation.random(random_state=rng).as_matrix()
    lo, hi = oracle.lattice_box((0, 0, 0), (0.4, 0.4, 0.4), delta)
    k, V, nb = oracle.vote(X, Y, R, delta, lo, hi)
    T = Y - R @ X[0]
    keys = [tuple(np.floor(tt / delta + 0.5).astype(int)) for tt in T]
    inbox = [kk for kk in keys if all(l <= a <= h for a, l, h in zip(kk, lo, hi))]
    assert len(set(inbox)) == len(inbox) and V == 1
    assert tuple(k) == min(inbox)


def test_vote_empty_box_gives_zero_votes_at_box_corner():
    X = np.zeros((3, 3))
    Y = np.array([[5.0, 5.0, 5.0], [6.0, 5.0, 5.0]])
    lo, hi = oracle.lattice_box((0, 0, 0), (0.2, 0.2, 0.2), 0.05)
    k, V, _ = oracle.vote(X, Y, np.eye(3), 0.05, lo, hi)
    assert V == 0 and k.tolist() == lo.tolist()


def test_vote_consistency_check_with_planted_boundary_pair():
    delta = 0.04
    X = np.zeros((1, 3))
    Y = np.array([[0.5 * delta - 1e-7, 0.0, 0.0], [1.0 * delta, 0.0, 0.0]])
    lo, hi = oracle.lattice_box((0, 0, 0), (0.2, 0.2, 0.2), delta)
    k, V, nb = oracle.vote(X, Y, np.eye(3), delta, lo, hi)
    assert k.tolist() == [0, 0, 0] and V == 1 and nb == 1
    assert oracle.vote_consistent(X, Y, np.eye(3), delta, lo, hi, [0, 0, 0], 1) == 2
    assert oracle.vote_consistent(X, Y, np.eye(3), delta, lo, hi, [1, 0, 0], 2) == 1
    assert oracle.vote_consistent(X, Y, np.eye(3), delta, lo, hi, [0, 0, 0], 2) == 0
    assert oracle.vote_consistent(X, Y, np.eye(3), delta, lo, hi, [2, 0, 0], 1) == 0
    # without the boundary pair nothing but the exact answer is consistent
    Y2 = np.array([[0.3 * delta, 0.0, 0.0], [1.0 * delta, 0.0, 0.0]])
    assert oracle.vote_consistent(X, Y2, np.eye(3), delta, lo, hi, [1, 0, 0], 2) == 0
    assert oracle.vote_consistent(X, Y2, np.eye(3), delta, lo, hi, [1, 0, 0], 1) == 0


def test_vote_translation_equivariance_on_dyadic_data():
    # Shifting the target by a lattice vector v = m delta (exactly representable)
    # and the search box by v shifts the mode by m and keeps V.
    rng = np.random.default_rng(11)
    delta = 2.0**-5
    X = synth.dyadic_cloud(rng, 20, extent=0.5)
    Y = synth.dyadic_cloud(rng, 30, extent=0.5)
    R = Rotation.random(random_state=rng).as_matrix()
    m = np.array([3, -2, 5])
    lo, hi = oracle.lattice_box((0, 0, 0), (0.6, 0.6, 0.6), delta)
    k, V, _ = oracle.vote(X, Y, R, delta, lo, hi)
    k2, V2, _ = oracle.vote(X, Y + m * delta, R, delta, lo + m, hi + m)
    assert V2 == V and (k2 - k).tolist() == m.tolist()


def test_vote_permutation_invariance():
    p = synth.tiny_problem(3)
    X, Y = p.X.astype(np.float64), p.Y.astype(np.float64)
    R = oracle.hopf_rotation(4, 1234)
    lo, hi = oracle.lattice_box(p.t_center, p.t_half, p.delta_t)
    rng = np.random.default_rng(0)
    a = oracle.vote(X, Y, R, p.delta_t, lo, hi)
    b = oracle.vote(X[rng.permutation(len(X))], Y[rng.permutation(len(Y))], R, p.delta_t, lo, hi)
    assert a[0].tolist() == b[0].tolist() and a[1] == b[1]


# ---------------------------------------------------------------------------
# nearest neighbours, inliers (Eq. 3), robust costs (Eq. 1)


def test_nn_inliers_and_exact_costs_match_kdtree():
    p = synth.modelnet_like_problem(2, m=400, hopf_n=2)
    X, Y = p.X.astype(np.float64), p.Y.astype(np.float64)
    R, t = p.R_true, p.t_true
    d = oracle.nn_dist(X, Y, R, t)
    ref, _ = cKDTree(Y).query(X @ R.T + t)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12)
    for eps in (0.01, 0.03, 0.05):
        M, nb = oracle.inliers(X, Y, R, t, eps)
        assert M == int((ref < eps).sum())
        assert nb == int((np.abs(ref - eps) <= 1e-5).sum())
    for metric, rho in [
        ("trunc_l1", lambda e: np.minimum(e, 0.05)),
        ("trunc_l2", lambda e: np.minimum(e, 0.05) ** 2),
        ("huber", lambda e: np.where(np.minimum(e, 0.05) <= 0.02, 0.5 * np.minimum(e, 0.05) ** 2,
                                     0.02 * (np.minimum(e, 0.05) - 0.01))),
        ("lp", lambda e: np.sqrt(e)),
        ("inlier", lambda e: (e >= 0.03).astype(float)),
    ]:
        P = oracle.make_params(metric=metric, epsilon=0.03, tau=0.05, huber_h=0.02, p=0.5)
        assert oracle.cost_exact(X, Y, R, t, P) == pytest.approx(float(rho(ref).sum()), rel=1e-12)


def test_rho_closed_forms():
    P = oracle.make_params(metric="huber", epsilon=0.01, tau=0.1, huber_h=0.02)
    assert oracle.rho(P, 0.01) == pytest.approx(0.5 * 0.01**2)
    assert oracle.rho(P, 0.04) == pytest.approx(0.02 * (0.04 - 0.01))
    assert oracle.rho(P, 5.0) == pytest.approx(0.02 * (0.1 - 0.01))
    P = oracle.make_params(metric="trunc_l2", epsilon=0.01, tau=0.1)
    assert oracle.rho(P, 0.05) == pytest.approx(0.0025) and oracle.rho(P, 3.0) == pytest.approx(0.01)
    P = oracle.make_params(metric="inlier", epsilon=0.01)
    assert oracle.rho(P, 0.00999) == 0.0 and oracle.rho(P, 0.01) == 1.0


def test_distance_grid_matches_kdtree_and_linear_interpolator():
    rng = np.random.default_rng(5)
    Y = rng.uniform(-0.5, 0.5, size=(60, 3))
    G, cap = 24, 0.15
    g = oracle.dist_grid(Y, G, cap)
    # geometry: outermost centres lie >= cap from every point
    ax = [g.lo[a] + (np.arange(G) + 0.5) * g.h[a] for a in range(3)]
    C = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
    dref, _ = cKDTree(Y).query(C)
    np.testing.assert_allclose(g.D.reshape(-1), np.minimum(dref, cap), atol=1e-12)
    assert np.all(g.D[0] == cap) and np.all(g.D[-1] == cap)
    assert np.all(g.D[:, 0] == cap) and np.all(g.D[:, :, -1] == cap)
    interp = RegularGridInterpolator(ax, g.D, method="linear")
    P = rng.uniform([a[0] for a in ax], [a[-1] for a in ax], size=(300, 3))
    got = np.array([oracle.grid_lookup(g, p) for p in P])
    np.testing.assert_allclose(got, interp(P), atol=1e-12)
    # outside the grid box: the cap; between the box face and the first centre:
    # clamped to the face centres (which hold the cap)
    assert oracle.grid_lookup(g, g.lo - 1e-3) == cap
    inner = g.lo + 0.25 * g.h
    assert oracle.grid_lookup(g, inner) == pytest.approx(cap)
    # grid cost = sum of rho over lookups
    X = rng.uniform(-0.4, 0.4, size=(25, 3))
    Pm = oracle.make_params(metric="trunc_l1", epsilon=0.02, tau=0.1)
    ref = sum(min(oracle.grid_lookup(g, x), 0.1) for x in X)
    assert oracle.cost_grid(X, g, np.eye(3), np.zeros(3), Pm) == pytest.approx(ref, rel=1e-12)


# ---------------------------------------------------------------------------
# Algorithm 2 end to end: the Theorem's special case and Algorithm 1


def _theorem_case(seed, n=2, N=24, M=60, delta=0.05):
    rng = np.random.default_rng(seed)
    Y = synth.dyadic_cloud(rng, M, extent=0.8, min_sep_inf=delta)
    grid = oracle.hopf_grid(n)
    r_true = int(rng.integers(len(grid)))
    R_true = grid[r_true]
    k_true = np.array([3, -4, 2])
    t_true = k_true * delta
    sub = Y[rng.choice(M, size=N, replace=False)]
    X = (sub - t_true) @ R_true  # x = R^T (y - t)
    return X, Y, grid, r_true, k_true, t_true


@pytest.mark.parametrize("seed", range(3))
def test_theorem_special_case_recovers_grid_pose(seed):
    X, Y, grid, r_true, k_true, t_true = _theorem_case(seed)
    for metric, nn in [("inlier", "grid"), ("trunc_l1", "brute"), ("trunc_l2", "grid")]:
        P = oracle.make_params(metric=metric, epsilon=0.05, tau=0.1, t_half=(0.5, 0.5, 0.5), nn_mode=nn,
                               grid_res=32)
        reg = oracle.register(X, Y, grid, P)
        assert reg.status == 0
        assert reg.rot_index == r_true
        np.testing.assert_allclose(reg.t, t_true, atol=1e-12)
        assert reg.votes == len(X) and reg.inliers == len(X)
        if metric == "inlier" or nn == "brute":
            assert reg.cost == pytest.approx(0.0, abs=1e-9)


def _exhaustive_inlier_max(X, Y, grid, delta, lo, hi):
    """Algorithm 1 restricted to the inlier metric on the delta lattice: for every
    rotation and every lattice translation, count source points with a target in
    the voxel of that translation (voxel-membership test)."""
    best = 0
    cells = np.array(list(itertools.product(*[range(l, h + 1) for l, h in zip(lo, hi)])))
    for R in grid:
        T = Y[None, :, :] - (X @ R.T)[:, None, :]  # (N, M, 3)
        key = np.floor(T / delta + 0.5).astype(np.int64)
        for c in cells:
            hit = np.all(key == c, axis=2).any(axis=1)
            best = max(best, int(hit.sum()))
    return best


def test_dses_max_votes_equals_exhaustive_inlier_optimum():
    # Theorem: with inf-norm separated targets, max over rotations of the vote
    # frequency equals Algorithm 1's inlier optimum over the same discretisation.
    rng = np.random.default_rng(21)
    delta = 0.1
    Y = synth.dyadic_cloud(rng, 18, extent=0.4, min_sep_inf=delta)
    X = synth.dyadic_cloud(rng, 7, extent=0.3)
    grid = oracle.hopf_grid(1)
    lo, hi = oracle.lattice_box((0, 0, 0), (0.3, 0.3, 0.3), delta)
    P = oracle.make_params(metric="inlier", epsilon=delta, t_half=(0.3, 0.3, 0.3))
    reg = oracle.register(X, Y, grid, P)
    assert int(reg.V.max()) == _exhaustive_inlier_max(X, Y, grid, delta, lo, hi)


def test_lemma_identity_votes_equal_points_with_a_target_in_the_mode_voxel():
    # Lemma 1's proof: with no two targets in one voxel window, each source point
    # supports the mode at most once, so V = #{i : some y_j in voxel k*} and the
    # saturated-L0 sum is N - V; with epsilon = delta every such point is an
    # inlier of Eq. 3 (its distance is at most sqrt(3)/2 delta).
    rng = np.random.default_rng(4)
    delta = 0.08
    Y = synth.dyadic_cloud(rng, 50, extent=0.6, min_sep_inf=delta)
    X = synth.dyadic_cloud(rng, 15, extent=0.4)
    grid = oracle.hopf_grid(1)
    P = oracle.make_params(metric="inlier", epsilon=delta, t_half=(0.5, 0.5, 0.5))
    reg = oracle.register(X, Y, grid, P)
    for r, R in enumerate(grid):
        c = reg.k[r] * delta
        T = Y[None, :, :] - (X @ R.T)[:, None, :]
        per_point = np.all((T >= c - delta / 2) & (T < c + delta / 2), axis=2).any(axis=1)
        assert reg.V[r] == int(per_point.sum())
        assert reg.M[r] >= reg.V[r]


def test_q_filter_and_top_k_selection():
    X, Y, grid, r_true, _, _ = _theorem_case(5, n=1)
    base = dict(metric="trunc_l1", epsilon=0.05, tau=0.1, t_half=(0.5, 0.5, 0.5), nn_mode="brute")
    reg_all = oracle.register(X, Y, grid, oracle.make_params(q_milli=0, **base))
    assert np.all(np.isfinite(reg_all.costs))
    reg_q = oracle.register(X, Y, grid, oracle.make_params(q_milli=500, **base))
    Mstar = reg_q.M.max()
    keep = 1000 * reg_q.M >= 500 * Mstar
    assert np.array_equal(np.isfinite(reg_q.costs), keep)
    reg_k = oracle.register(X, Y, grid, oracle.make_params(top_k=5, **base))
    order = sorted(range(len(grid)), key=lambda r: (-reg_k.M[r], r))[:5]
    assert sorted(np.flatnonzero(np.isfinite(reg_k.costs)).tolist()) == sorted(order)
    for reg in (reg_all, reg_q, reg_k):
        assert reg.rot_index == r_true


def test_refinement_pass_indices_and_monotonicity():
    p = synth.tiny_problem(1, hopf_n=1)
    grid = oracle.hopf_grid(1)
    P0 = oracle.params_from_problem(p, nn_mode="brute")
    P1 = oracle.params_from_problem(p, nn_mode="brute", refine_top_k=4, refine_K=1,
                                    refine_delta_r=math.radians(5))
    a = oracle.register(p.X, p.Y, grid, P0)
    b = oracle.register(p.X, p.Y, grid, P1)
    assert len(b.V) == len(grid) + 4 * 27
    np.testing.assert_array_equal(a.V, b.V[: len(grid)])
    assert b.cost <= a.cost
    # the centre sample of each local box (zero Euler angles: the centre
    # rotation itself) has the outputs of the c-th best coarse candidate by
    # (cost, index); the four candidates differ, so a box around the wrong
    # candidate shows
    order = sorted(np.flatnonzero(np.isfinite(a.costs)), key=lambda r: (a.costs[r], r))[:4]
    outs = [(tuple(a.k[r]), a.V[r], a.M[r], a.costs[r]) for r in order]
    assert len(set(outs)) == len(outs)
    for c, r in enumerate(order):
        f = len(grid) + c * 27 + 13
        assert (tuple(b.k[f]), b.V[f], b.M[f], b.costs[f]) == outs[c], c


def test_inlier_threshold_is_strict():
    # Eq. 3 read with a strict tolerance: a point exactly epsilon away is an
    # outlier (dyadic values, so the distance is exact).
    X = np.zeros((2, 3))
    Y = np.array([[0.25, 0.0, 0.0], [5.0, 5.0, 5.0]])
    assert oracle.inliers(X[:1], Y, np.eye(3), np.zeros(3), 0.25)[0] == 0
    assert oracle.inliers(X[:1], Y, np.eye(3), np.zeros(3), 0.25 + 2**-20)[0] == 1


def test_exhaustive_inlier_threshold_is_strict():
    # Algorithm 1's count and the inlier metric take the same strict reading:
    # at the one lattice translation t = 0, the source point lies exactly
    # epsilon from its target (dyadic values, exact distance)
    X = np.zeros((1, 3))
    Y = np.array([[0.25, 0.0, 0.0], [5.0, 5.0, 5.0]])
    for eps, n_in in ((0.25, 0), (0.25 + 2**-20, 1)):
        P = oracle.make_params(metric="inlier", epsilon=eps, delta_t=0.25, t_half=(0.0, 0.0, 0.0))
        cost, cnt, best, _ = oracle.exhaustive(X, Y, np.eye(3)[None], P)
        assert cnt.shape == (1, 1) and cnt[0, 0] == n_in and cost[0, 0] == 1 - n_in


def test_q_filter_keeps_equality():
    # q = 1 keeps exactly the rotations with M = M* (Algorithm 2's "M >= q M*").
    X, Y, grid, r_true, _, _ = _theorem_case(6, n=1)
    P = oracle.make_params(metric="trunc_l1", epsilon=0.05, tau=0.1, t_half=(0.5, 0.5, 0.5), nn_mode="brute",
                           q_milli=1000)
    reg = oracle.register(X, Y, grid, P)
    keep = reg.M == reg.M.max()
    assert np.array_equal(np.isfinite(reg.costs), keep) and reg.rot_index == r_true


def test_selection_on_planted_inlier_counts():
    # Candidate selection against counts fixed by construction, not by the
    # oracle's own arithmetic: X = Y holds 3 points on the z axis and 7 points
    # off it; a rotation about z by 180 or 90 degrees leaves only the axis
    # points on targets (the others land far from every target and outside the
    # +-delta translation box), the identity leaves all 10. Grid [Rz180, I,
    # Rz90, I, Rz180] therefore has M = [3, 10, 3, 10, 3], M* = 10, and:
    # q = 0.3 keeps every rotation (1000 * 3 == 300 * 10: the filter is >=);
    # q = 0.301 keeps the two identities; top-3 by (M desc, index asc) is
    # {1, 3, 0}; the best (inlier metric, cost N - M) is rotation 1.
    delta = 0.05
    axis = np.array([[0.0, 0.0, -0.4], [0.0, 0.0, 0.1], [0.0, 0.0, 0.45]])
    off = np.array([[0.7, 0.1, 0.0], [0.3, 0.9, 0.2], [-0.2, 0.6, -0.3], [0.5, -0.8, 0.4],
                    [0.9, 0.4, -0.6], [0.15, -0.35, 0.7], [-0.55, -0.2, 0.25]])
    Y = np.vstack([axis, off])
    X = Y.copy()
    Rz = lambda deg: Rotation.from_euler("z", deg, degrees=True).as_matrix()
    grid = np.stack([Rz(180), np.eye(3), Rz(90), np.eye(3), Rz(180)])
    # the construction: rotated off-axis points are far from every target
    for R in (Rz(180), Rz(90)):
        d = np.linalg.norm((off @ R.T)[:, None, :] - Y[None, :, :], axis=2)
        assert d.min() > 4 * delta
    want_M = [3, 10, 3, 10, 3]
    base = dict(metric="inlier", epsilon=delta, t_half=(delta, delta, delta), nn_mode="brute")
    for q, kept in ((0, [0, 1, 2, 3, 4]), (300, [0, 1, 2, 3, 4]), (301, [1, 3]), (1000, [1, 3])):
        reg = oracle.register(X, Y, grid, oracle.make_params(q_milli=q, **base))
        assert reg.M.tolist() == want_M and reg.V.tolist() == want_M
        assert np.flatnonzero(np.isfinite(reg.costs)).tolist() == kept, q
        assert reg.rot_index == 1 and reg.inliers == 10
    reg = oracle.register(X, Y, grid, oracle.make_params(top_k=3, **base))
    assert sorted(np.flatnonzero(np.isfinite(reg.costs)).tolist()) == [0, 1, 3]
    reg = oracle.register(X, Y, grid, oracle.make_params(top_k=1, **base))
    assert np.flatnonzero(np.isfinite(reg.costs)).tolist() == [1]


# ---------------------------------------------------------------------------
# sub-voxel translation refinement (mean of the inlier translations)


def _separated_cloud(rng, m, spacing):
    """m points of a jittered cubic lattice: every pair at least `spacing` apart."""
    side = int(math.ceil(m ** (1 / 3))) + 1
    cells = np.array(list(itertools.product(range(side), repeat=3)), float)
    pick = cells[rng.choice(len(cells), m, replace=False)]
    return (pick + rng.uniform(-0.2, 0.2, pick.shape)) * spacing


def test_refine_translation_recovers_exact_pose_on_noiseless_subset():
    # X is an exact subset of Y moved by (R, t): from any start within a
    # quarter of the spacing every source point pairs with its own target, so
    # the mean of the inlier translations is t itself.
    rng = np.random.default_rng(3)
    Y = _separated_cloud(rng, 300, 0.1)
    R = Rotation.random(random_state=4).as_matrix()
    t = np.array([0.31, -0.12, 0.07])
    Xs = Y[rng.choice(300, 120, replace=False)]
    X = (Xs - t) @ R  # rows: R^T (y - t)
    start = t + np.array([0.012, -0.009, 0.014])
    tr, n, nb, nt = oracle.refine_translation(X, Y, R, start, eps=0.04)
    assert n == 120 and nb == 0 and nt == 0
    np.testing.assert_allclose(tr, t, atol=1e-12)


def test_refine_translation_is_the_least_squares_translation_of_the_inliers():
    # Correspondences from cKDTree at the start pose, inliers below epsilon;
    # the refined t must be the least-squares solution of
    # min_t sum_i ||y_nn(i) - R x_i - t||^2 over those inliers (numpy lstsq on
    # the stacked identity design), with clutter points excluded.
    rng = np.random.default_rng(5)
    Y = _separated_cloud(rng, 400, 0.1)
    R = Rotation.random(random_state=6).as_matrix()
    t = np.array([-0.2, 0.4, 0.1])
    Xs = Y[rng.choice(400, 150, replace=False)] + rng.normal(0, 0.004, (150, 3))
    clutter = rng.uniform(-2, 3, (40, 3))
    X = (np.vstack([Xs, clutter]) - t) @ R
    start = t + np.array([0.01, 0.008, -0.006])
    eps = 0.035
    tr, n, nb, nt = oracle.refine_translation(X, Y, R, start, eps=eps)
    assert nb == 0 and nt == 0
    U = X @ R.T
    dist, idx = cKDTree(Y).query(U + start)
    keep = dist < eps
    assert n == int(keep.sum()) and 140 <= n <= 150
    A = np.tile(np.eye(3), (n, 1))
    b = (Y[idx[keep]] - U[keep]).reshape(-1)
    ls = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(tr, ls, atol=1e-12)
    assert np.linalg.norm(tr - t) < np.linalg.norm(start - t)


def test_refine_translation_equivariance_and_no_inlier_case():
    rng = np.random.default_rng(7)
    Y = _separated_cloud(rng, 200, 0.1)
    R = Rotation.random(random_state=8).as_matrix()
    X = (Y[:80] + rng.normal(0, 0.003, (80, 3))) @ R
    start = np.array([0.004, -0.006, 0.002])
    v = np.array([1.25, -0.5, 0.75])
    a, na, _, _ = oracle.refine_translation(X, Y, R, start, eps=0.03)
    b, nb_, _, _ = oracle.refine_translation(X, Y + v, R, start + v, eps=0.03)
    assert na == nb_ == 80
    np.testing.assert_allclose(b, a + v, atol=1e-12)
    far = np.array([50.0, 0.0, 0.0])
    c, nc, _, _ = oracle.refine_translation(X, Y, R, far, eps=0.03)
    assert nc == 0
    np.testing.assert_array_equal(c, far)


# ---------------------------------------------------------------------------
# Algorithm 1 (pure exhaustive search)


def _tiny_pose_problem(seed, n_src=9, n_tgt=20, delta=0.1, K=1):
    rng = np.random.default_rng(seed)
    Y = synth.dyadic_cloud(rng, n_tgt, extent=0.4, min_sep_inf=delta)
    rots = oracle.euler_box(np.eye(3), K, math.radians(20.0))
    return rng, Y, rots


@pytest.mark.parametrize("metric", ["inlier", "trunc_l1", "trunc_l2", "huber", "lp"])
def test_exhaustive_matches_numpy_brute_force(metric):
    # every (rotation, lattice translation) entry against cKDTree distances and
    # the closed-form rho, in the stated index order
    rng, Y, rots = _tiny_pose_problem(2)
    X = rng.uniform(-0.3, 0.3, (9, 3))
    P = oracle.make_params(metric=metric, epsilon=0.1, tau=0.15, huber_h=0.05, p=0.5, t_half=(0.2, 0.2, 0.2))
    cost, cnt, best, _ = oracle.exhaustive(X, Y, rots, P)
    lo, hi = oracle.lattice_box((0, 0, 0), (0.2, 0.2, 0.2), 0.1)
    ks = list(itertools.product(*[range(a, b + 1) for a, b in zip(lo, hi)]))
    assert cost.shape == (len(rots), len(ks))
    tree = cKDTree(Y)
    for r, R in enumerate(rots):
        for ti, k in enumerate(ks):
            d, _ = tree.query(X @ R.T + np.array(k) * 0.1)
            e = np.minimum(d, 0.15)
            ref = {"inlier": float(np.sum(d >= 0.1)), "trunc_l1": e.sum(), "trunc_l2": (e * e).sum(),
                   "huber": np.where(e <= 0.05, 0.5 * e * e, 0.05 * (e - 0.025)).sum(),
                   "lp": np.sqrt(d).sum()}[metric]
            assert abs(cost[r, ti] - ref) <= 1e-9 * max(1.0, abs(ref))
            assert cnt[r, ti] == int(np.sum(d < 0.1))
    assert best == int(np.argmin(cost.reshape(-1)))


def test_exhaustive_finds_the_planted_pose_with_zero_error():
    # Theorem setting: the source is a subset of the target moved by a grid
    # rotation and a lattice translation; only that entry has zero error
    rng, Y, rots = _tiny_pose_problem(4)
    r_true, k_true = 17, np.array([1, -1, 0])
    R = rots[r_true]
    X = (Y[:8] - k_true * 0.1) @ R  # rows R^T (y - t)
    P = oracle.make_params(metric="trunc_l1", epsilon=0.1, tau=0.15, t_half=(0.2, 0.2, 0.2))
    cost, cnt, best, _ = oracle.exhaustive(X, Y, rots, P)
    lo, hi = oracle.lattice_box((0, 0, 0), (0.2, 0.2, 0.2), 0.1)
    E = hi - lo + 1
    ti = ((k_true[0] - lo[0]) * E[1] + (k_true[1] - lo[1])) * E[2] + (k_true[2] - lo[2])
    assert best == r_true * cost.shape[1] + ti
    assert cost.reshape(-1)[best] < 1e-12 and cnt.reshape(-1)[best] == 8
    assert np.sort(cost.reshape(-1))[1] > 1e-3


def test_dses_per_rotation_cost_is_the_exhaustive_entry_at_its_mode():
    # Algorithm 2 evaluates each rotation at its vote mode t*: with exact nearest
    # neighbours its per-rotation cost and inlier count are Algorithm 1's entry
    # at (r, t*), and so its best cost is never below Algorithm 1's optimum
    rng, Y, rots = _tiny_pose_problem(6)
    X = (Y[:8] + rng.normal(0, 0.01, (8, 3)) - np.array([0.1, 0.0, -0.1])) @ rots[5]
    P = oracle.make_params(metric="trunc_l2", epsilon=0.1, tau=0.15, t_half=(0.2, 0.2, 0.2), nn_mode="brute")
    cost, cnt, best, _ = oracle.exhaustive(X, Y, rots, P)
    reg = oracle.register(X, Y, rots, P)
    lo, hi = oracle.lattice_box((0, 0, 0), (0.2, 0.2, 0.2), 0.1)
    E = hi - lo + 1
    for r in range(len(rots)):
        k = reg.k[r]
        ti = ((k[0] - lo[0]) * E[1] + (k[1] - lo[1])) * E[2] + (k[2] - lo[2])
        assert abs(reg.costs[r] - cost[r, ti]) <= 1e-12
        assert reg.M[r] == cnt[r, ti]
    assert reg.cost >= cost.reshape(-1)[best] - 1e-12


def test_refine_translation_inlier_threshold_is_strict_and_tight():
    # source points displaced from their own target by 0.9 eps count, those
    # displaced by 1.1 eps do not (targets are 0.1 apart, so the nearest target
    # is always the own one); the mean then uses the 0.9 eps points only
    rng = np.random.default_rng(11)
    Y = _separated_cloud(rng, 200, 0.1)
    eps = 0.02
    dirs = rng.normal(size=(60, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    scale = np.where(np.arange(60) < 35, 0.9 * eps, 1.1 * eps)[:, None]
    X = Y[:60] - dirs * scale  # R = I, t = 0: y - x = dirs * scale
    tr, n, nb, nt = oracle.refine_translation(X, Y, np.eye(3), np.zeros(3), eps)
    assert n == 35 and nb == 0 and nt == 0
    np.testing.assert_allclose(tr, (dirs[:35] * 0.9 * eps).mean(axis=0), atol=1e-15)
