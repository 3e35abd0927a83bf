"""The parity harness (tests/parity.py) itself, on the CPU: fed the oracle's
own per-rotation outputs it passes every rotation exactly, and each kind of
planted error in a "GPU" output (a vote count, a mode index, an inlier count,
a cost beyond the tolerance, a wrong best rotation) is reported, so the GPU
parity tests cannot pass vacuously."""
import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import synth
from parity import check_rotations, result_matches_oracle


@pytest.fixture(scope="module")
def case():
    p = synth.tiny_problem(3, hopf_n=1)
    grid = oracle.hopf_grid(1)
    P = oracle.params_from_problem(p, nn_mode="brute")
    ref = oracle.register(p.X, p.Y, grid, P)
    return p, grid, P, ref, int(np.argmax(ref.V))


def _outputs(ref):
    return ref.k.copy(), ref.V.copy(), ref.M.copy(), ref.costs.copy()


def test_oracle_outputs_pass_exactly(case):
    p, grid, P, ref, _ = case
    k, V, M, C = _outputs(ref)
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, range(len(grid)), ref=ref)
    assert rep.ok() and rep.vote_exact == rep.m_exact == rep.cost_checked == len(grid), rep.summary()
    # the same without the stored reference (each rotation re-evaluated)
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, [0, 5, 71])
    assert rep.ok() and rep.vote_exact == 3, rep.summary()
    # a cost inside the tolerance passes
    C2 = C.copy()
    C2[0] *= 1 + 1e-6
    assert check_rotations(p.X, p.Y, grid, P, k, V, M, C2, [0], ref=ref).ok()


@pytest.mark.parametrize("kind", ["votes", "mode", "inliers", "cost"])
def test_planted_errors_are_reported(case, kind):
    # each error is the smallest the rules cannot excuse at that rotation:
    # every boundary pair can add at most one vote to a voxel and every
    # boundary point change M by one
    p, grid, P, ref, r = case
    k, V, M, C = _outputs(ref)
    if kind == "votes":
        V[r] += ref.n_boundary_pairs[r] + 1
    elif kind == "mode":
        k[r, 0] += 20
    elif kind == "inliers":
        M[r] += ref.n_boundary_points[r] + 1
    else:
        C[r] *= 1 + 1e-3
    rep = check_rotations(p.X, p.Y, grid, P, k, V, M, C, range(len(grid)), ref=ref)
    assert not rep.ok()
    tag = {"votes": "vote", "mode": "vote", "inliers": "inliers", "cost": "cost"}[kind]
    assert [f[:2] for f in rep.failures] == [(tag, r)], rep.failures


def test_result_check_rejects_a_worse_rotation(case):
    p, grid, P, ref, _ = case
    res = {"status": 0, "rot_index": ref.rot_index, "votes": ref.votes, "inliers": ref.inliers, "t": ref.t,
           "cost": ref.cost}
    result_matches_oracle(res, ref, len(p.X))
    worst = int(np.argmax(ref.costs))
    assert ref.costs[worst] > 1.01 * ref.cost
    bad = dict(res, rot_index=worst, cost=ref.costs[worst])
    with pytest.raises(AssertionError):
        result_matches_oracle(bad, ref, len(p.X))
    with pytest.raises(AssertionError):
        result_matches_oracle(dict(res, cost=ref.cost * 1.01), ref, len(p.X))
