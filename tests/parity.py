"""Per-rotation parity of the CUDA path against the FP64 oracle.

FP32 and FP64 may only decide differently where a value sits within the
boundary band (1e-5) of a decision threshold: a point pair within the band of
a voxel face, or a source point whose nearest-target distance is within the
band of epsilon. The rules:

* vote: (k*, V) equal to the oracle's, or "consistent" -- achievable when
  every boundary pair may land in any voxel it is within the band of
  (oracle.vote_consistent); anything else fails;
* inliers: the oracle recounts M at the GPU's t*; |dM| must not exceed that
  rotation's boundary points;
* cost: the oracle rescored at the GPU's (R, t*) with the same
  nearest-neighbour definition (exact or the distance grid); relative error
  <= 1e-4 (absolute floor 1e-6 per source point);
* best rotation: equal, or a near-tie whose oracle costs agree within 1e-4.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

COST_RTOL = 1e-4


@dataclasses.dataclass
class Report:
    checked: int = 0
    vote_exact: int = 0
    vote_excused: int = 0
    m_exact: int = 0
    m_excused: int = 0
    cost_checked: int = 0
    max_cost_rel: float = 0.0
    failures: list = dataclasses.field(default_factory=list)

    def ok(self):
        return not self.failures

    def summary(self):
        return (f"checked={self.checked} vote exact={self.vote_exact} excused={self.vote_excused} "
                f"M exact={self.m_exact} excused={self.m_excused} cost checked={self.cost_checked} "
                f"max rel={self.max_cost_rel:.2e} failures={self.failures[:5]}")


def cost_close(got, ref, n):
    return abs(float(got) - float(ref)) <= COST_RTOL * abs(float(ref)) + 1e-6 * n


def check_rotations(X, Y, rotations64, P, k_gpu, V_gpu, M_gpu, cost_gpu, indices, ref=None, dist_grid=None,
                    rep: Report | None = None) -> Report:
    """Check the GPU's per-rotation outputs at `indices` (global rotation indices).

    rotations64[i] is the oracle's FP64 rotation for indices[i] (or for every
    index when it covers them all); ref: an oracle Registration with per-rotation
    arrays for the same indices (optional: recomputed otherwise)."""
    rep = rep or Report()
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    for pos, r in enumerate(indices):
        R = rotations64[pos] if len(rotations64) == len(indices) else rotations64[r]
        rep.checked += 1
        if ref is not None:
            k_o, V_o = ref.k[r], ref.V[r]
        else:
            k_o, V_o, _, _, _ = oracle.eval_rotation(X, Y, R, P)
        kg = np.asarray(k_gpu[r], dtype=np.int64)
        if np.array_equal(kg, k_o) and int(V_gpu[r]) == int(V_o):
            rep.vote_exact += 1
        else:
            c = oracle.vote_consistent(X, Y, R, P.delta_t, lo, hi, kg, int(V_gpu[r]), band=P.band)
            if c == 0:
                rep.failures.append(("vote", int(r), kg.tolist(), int(V_gpu[r]), np.asarray(k_o).tolist(), int(V_o)))
                continue
            rep.vote_excused += 1
        t = kg * float(P.delta_t)
        M_o, nb = oracle.inliers(X, Y, R, t, P.epsilon, band=P.band)
        dM = abs(int(M_gpu[r]) - M_o)
        if dM == 0:
            rep.m_exact += 1
        elif dM <= nb:
            rep.m_excused += 1
        else:
            rep.failures.append(("inliers", int(r), int(M_gpu[r]), M_o, nb))
            continue
        if cost_gpu is not None and np.isfinite(cost_gpu[r]):
            if P.metric == 0:
                c_ref = len(X) - int(M_gpu[r])
            elif P.nn_mode == 1:
                c_ref = oracle.cost_exact(X, Y, R, t, P)
            else:
                c_ref = oracle.cost_grid(X, dist_grid, R, t, P)
            rep.cost_checked += 1
            rel = abs(float(cost_gpu[r]) - c_ref) / max(abs(c_ref), 1e-12)
            rep.max_cost_rel = max(rep.max_cost_rel, rel)
            if not cost_close(cost_gpu[r], c_ref, len(X)):
                rep.failures.append(("cost", int(r), float(cost_gpu[r]), c_ref))
    return rep


def best_matches(gpu_best: int, ref, costs_oracle_at=None) -> bool:
    """Exact best index, or a near-tie: the oracle's costs of both indices agree."""
    if gpu_best == ref.rot_index:
        return True
    if costs_oracle_at is None:
        return False
    a, b = costs_oracle_at(gpu_best), costs_oracle_at(ref.rot_index)
    return cost_close(a, b, 1)


def result_matches_oracle(res: dict, ref, n_src: int) -> None:
    """A registration's result against the oracle's registration of the same
    problem: the best index equal (then V and M equal, unless that rotation has
    boundary pairs or points, and t* equal unless it has boundary pairs), or a
    near-tie of the oracle's costs; the cost within the cost tolerance of the
    oracle's cost at the returned rotation."""
    r = int(res["rot_index"])
    assert res["status"] == 0 == ref.status, (res["status"], ref.status)
    if r == ref.rot_index:
        nbp, nbm = int(ref.n_boundary_pairs[r]), int(ref.n_boundary_points[r])
        assert res["votes"] == ref.votes or nbp > 0, (res["votes"], ref.votes)
        assert res["inliers"] == ref.inliers or nbm > 0 or nbp > 0, (res["inliers"], ref.inliers)
        assert np.allclose(res["t"], ref.t, atol=1e-6) or nbp > 0, (res["t"], ref.t)
    else:
        assert cost_close(ref.costs[r], ref.costs[ref.rot_index], 1), (r, ref.rot_index)
    assert cost_close(res["cost"], ref.costs[r], n_src), (res["cost"], ref.costs[r])
