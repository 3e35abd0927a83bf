"""Oracle parity of every benchmark configuration at its own size and in the
launch configuration the benchmark times:

* ModelNet-shaped single problem (294,912 rotations, 717 x 1,024 points):
  every rotation's (k*, V, M, cost) and the best index against the stored
  FP64 oracle values (tests/golden/make_modelnet_like_golden.py);
* batched: the 64 uneven problems in one persistent launch, sampled
  rotations and every problem's winner against the oracle;
* serving: requests of the serving workload (16 resident targets, N_side 10,
  lognormal source sizes) submitted at their Poisson arrival times; each
  served result equals the same problem registered alone and its winner,
  with sampled rotations, agrees with the oracle;
* robot-pose-like (2.36M rotations + Euler boxes around the best 32, 5,000 x
  20,000 points, Huber): sampled first- and second-pass rotations with their
  costs, the second pass's boxes rebuilt by the oracle around the GPU's
  chosen centres.

Rules as in tests/parity.py: integer outputs exact unless a boundary pair or
point (within 1e-5 of a decision) excuses them, costs within 1e-4 relative.
"""
import concurrent.futures as cf
import hashlib
import os
import time

import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import build, capi, synth
from parity import Report, check_rotations, cost_close
from test_gpu_parity import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden", "modelnet_like_nside16_seed0.npz")
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = capi.Context(0)
    yield c
    c.close()


def parallel(fn, items):
    """fn over items on all host threads (the oracle's ctypes calls release the GIL)."""
    with cf.ThreadPoolExecutor(max_workers=THREADS) as ex:
        return list(ex.map(fn, items))


def check_parallel(X, Y, Rs, P, k, V, M, C, idx, dist_grid=None) -> Report:
    """check_rotations over idx, split across host threads, reports merged."""
    chunks = [list(range(i, len(idx), THREADS)) for i in range(min(THREADS, len(idx)))]

    def one(ch):
        return check_rotations(X, Y, [Rs[i] for i in ch], P, k, V, M, C, [idx[i] for i in ch], dist_grid=dist_grid)

    rep = Report()
    for r in parallel(one, chunks):
        for f in ("checked", "vote_exact", "vote_excused", "m_exact", "m_excused", "cost_checked"):
            setattr(rep, f, getattr(rep, f) + getattr(r, f))
        rep.max_cost_rel = max(rep.max_cost_rel, r.max_cost_rel)
        rep.failures += r.failures
    return rep


def argmin_cost(C):
    """The kernels' argmin order over (cost, index), NaN (not a candidate) last."""
    c = np.where(np.isfinite(C), C, np.inf)
    return int(np.lexsort((np.arange(len(c)), c))[0])


# ---------------------------------------------------------------------------
# ModelNet-shaped problem, every rotation


def test_modelnet_like_every_rotation_matches_stored_oracle(ctx):
    if not os.path.exists(GOLD):
        pytest.fail(f"{GOLD} is missing: run tests/golden/make_modelnet_like_golden.py")
    g = np.load(GOLD)
    p = synth.modelnet_like_problem(0)
    digest = lambda a: hashlib.sha256(np.ascontiguousarray(a, dtype=np.float32).tobytes()).hexdigest()
    assert digest(p.X) == str(g["x_sha256"]) and digest(p.Y) == str(g["y_sha256"]), "the generator changed"
    cap = 2 * p.tau
    t = ctx.create_target(p.Y, grid_cap=cap)
    gp = gpu_params(p, nn_mode="grid")
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gp)
    n = 72 * p.hopf_n**3
    k, V, M, C, r = ctx.debug(pb, n)
    ctx.destroy_target(t)
    P = oracle_params(p, gp, cap)
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    k_o = g["k_rel"].astype(np.int64) + g["lo"].astype(np.int64)[None, :]
    V_o, M_o = g["V"].astype(np.int64), g["M"].astype(np.int64)
    C_o, nbm = g["cost"].astype(np.float64), g["n_boundary_points"].astype(np.int64)
    vote_same = np.all(k == k_o, axis=1) & (V.astype(np.int64) == V_o)
    bad_vote = np.nonzero(~vote_same)[0]

    def excuse_vote(r_):
        R = oracle.hopf_rotation(p.hopf_n, int(r_))
        ok = oracle.vote_consistent(p.X, p.Y, R, P.delta_t, lo, hi, k[r_], int(V[r_])) > 0
        m_o, nb = oracle.inliers(p.X, p.Y, R, k[r_] * P.delta_t, P.epsilon)
        return ok, abs(int(M[r_]) - m_o) <= nb

    checks = parallel(excuse_vote, bad_vote)
    assert all(v for v, _ in checks), [int(r_) for r_, (v, _) in zip(bad_vote, checks) if not v][:10]
    assert all(m for _, m in checks)
    # M where the translation agrees: equal, or within the boundary points
    dM = np.abs(M.astype(np.int64) - M_o)
    m_bad = vote_same & (dM > nbm)
    assert not m_bad.any(), np.nonzero(m_bad)[0][:10]
    # costs where the translation agrees (the stored FP64 cost at the same pose)
    tol = 1e-4 * np.abs(C_o) + 1e-6 * len(p.X)
    c_bad = vote_same & ~(np.abs(C.astype(np.float64) - C_o) <= tol)
    assert not c_bad.any(), [(int(i), float(C[i]), float(C_o[i])) for i in np.nonzero(c_bad)[0][:10]]
    if len(bad_vote):  # costs at the GPU's own translation, rescored by the oracle
        dg = oracle.dist_grid(p.Y, 128, P.grid_cap, threads=THREADS)
        for r_ in bad_vote:
            c_ref = oracle.cost_grid(p.X, dg, oracle.hopf_rotation(p.hopf_n, int(r_)), k[r_] * P.delta_t, P)
            assert cost_close(C[r_], c_ref, len(p.X)), (int(r_), float(C[r_]), c_ref)
    # the best rotation: the oracle's, or a near-tie of its costs
    best = int(g["best"])
    assert r.status == 0 and r.rot_index == argmin_cost(C)
    assert r.rot_index == best or cost_close(C_o[r.rot_index], C_o[best], 1), (r.rot_index, best)
    rel = np.abs(C.astype(np.float64) - C_o)[vote_same] / np.maximum(np.abs(C_o[vote_same]), 1e-12)
    print(f"parity modelnet_like N_side 16: {n} rotations, (k*, V) exact {int(vote_same.sum())}, excused "
          f"{len(bad_vote)}; M exact {int((dM == 0).sum())}, excused {int(((dM > 0) & (dM <= nbm)).sum())}; "
          f"max cost rel {rel.max():.2e}; best {r.rot_index} (oracle {best})")


# ---------------------------------------------------------------------------
# 64 uneven problems in one persistent launch


def test_batched_64_problems_match_oracle(ctx):
    probs = synth.batch_problems(0, count=64)
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    gps = [gpu_params(p, nn_mode="grid") for p in probs]
    pbs = [ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gp) for t, p, gp in zip(targets, probs, gps)]
    n_rots = [72 * p.hopf_n**3 for p in probs]
    k, V, M, C, res = ctx.debug_batch(pbs, n_rots)
    for t in targets:
        ctx.destroy_target(t)
    # every problem's result is the argmin of its own per-rotation costs
    for b in range(len(probs)):
        w = argmin_cost(C[b])
        assert res[b].status == 0 and res[b].rot_index == w, b
        assert res[b].votes == V[b][w] and res[b].inliers == M[b][w] and res[b].cost == C[b][w]
    # sampled rotations and the winner of every problem against the oracle;
    # costs on the oracle's own distance grid for a quarter of the problems
    rng = np.random.default_rng(3)
    with_cost = set(rng.choice(len(probs), size=16, replace=False).tolist())
    grids = dict(zip(sorted(with_cost), parallel(
        lambda b: oracle.dist_grid(probs[b].Y, 128, float(np.float32(2 * probs[b].tau))), sorted(with_cost))))
    total = Report()
    for b, p in enumerate(probs):
        P = oracle_params(p, gps[b], 2 * p.tau)
        idx = sorted(set(rng.choice(n_rots[b], size=20, replace=False).tolist()) | {int(res[b].rot_index)})
        Rs = [oracle.hopf_rotation(p.hopf_n, i) for i in idx]
        rep = check_parallel(p.X, p.Y, Rs, P, k[b], V[b], M[b], C[b] if b in with_cost else None, idx,
                             dist_grid=grids.get(b))
        assert rep.ok(), (b, rep.summary())
        for f in ("checked", "vote_exact", "vote_excused", "m_exact", "m_excused", "cost_checked"):
            setattr(total, f, getattr(total, f) + getattr(rep, f))
        total.max_cost_rel = max(total.max_cost_rel, rep.max_cost_rel)
    print("parity batched (64 problems):", total.summary())


# ---------------------------------------------------------------------------
# served requests of the serving workload


def test_serving_workload_requests_match_oracle_and_solo(ctx):
    wl = synth.serving_workload(0, rate=200.0, duration=0.12)  # ~24 requests, 16 resident targets
    targets = [ctx.create_target(Y, grid_cap=0.1) for Y in wl.targets]
    pbs, gps = [], []
    for (_, ti, p) in wl.requests:
        gp = gpu_params(p, nn_mode="grid")
        gps.append(gp)
        pbs.append(ctx.problem(targets[ti], p.X, capi.hopf_grid(p.hopf_n), gp))
    for ti in sorted({ti for _, ti, _ in wl.requests}):  # warm each target's structures
        first = next(i for i, (_, t2, _) in enumerate(wl.requests) if t2 == ti)
        ctx.register(pbs[first])
    ctx.set_option("serve_max_active", 0)
    tickets, t0 = [], time.perf_counter()
    for (arr, _, _), pb in zip(wl.requests, pbs):
        while time.perf_counter() - t0 < arr:
            time.sleep(0.0005)
        tickets.append(ctx.submit(pb))
    served, deadline = {}, time.time() + 300
    while len(served) < len(tickets) and time.time() < deadline:
        for tk in tickets:
            if tk not in served:
                st, r = ctx.poll(tk)
                if st != capi.DSES_NOT_READY:
                    assert st == capi.DSES_OK
                    served[tk] = capi.result_dict(r)
        time.sleep(0.001)
    assert len(served) == len(tickets)
    assert ctx.get_option("serve_max_active") >= 2  # requests overlapped on the device
    rng = np.random.default_rng(4)
    grids = {}
    used = sorted({ti for _, ti, _ in wl.requests})
    for ti, g in zip(used, parallel(lambda ti: oracle.dist_grid(wl.targets[ti], 128, float(np.float32(0.1))), used)):
        grids[ti] = g
    total = Report()
    for (tk, pb, gp, (_, ti, p)) in zip(tickets, pbs, gps, wl.requests):
        n = 72 * p.hopf_n**3
        k, V, M, C, r = ctx.debug(pb, n)  # the same problem alone
        a, b = served[tk], capi.result_dict(r)
        assert a["rot_index"] == b["rot_index"] and a["inliers"] == b["inliers"] and a["votes"] == b["votes"]
        assert np.array_equal(a["t"], b["t"]) and a["cost"] == b["cost"]
        assert a["rot_index"] == argmin_cost(C)
        P = oracle_params(p, gp, 0.1)
        idx = sorted(set(rng.choice(n, size=8, replace=False).tolist()) | {a["rot_index"]})
        Rs = [oracle.hopf_rotation(p.hopf_n, i) for i in idx]
        rep = check_parallel(p.X, p.Y, Rs, P, k, V, M, C, idx, dist_grid=grids[ti])
        assert rep.ok(), (tk, rep.summary())
        for f in ("checked", "vote_exact", "vote_excused", "m_exact", "m_excused", "cost_checked"):
            setattr(total, f, getattr(total, f) + getattr(rep, f))
        total.max_cost_rel = max(total.max_cost_rel, rep.max_cost_rel)
    print(f"parity serving ({len(tickets)} requests):", total.summary())
    for t in targets:
        ctx.destroy_target(t)


# ---------------------------------------------------------------------------
# robot-pose-like problem: both passes, with costs


def test_robot_like_first_and_second_pass_with_costs(ctx):
    p = synth.robot_like_problem(0)
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    gp = gpu_params(p, nn_mode="grid", huber_h=p.huber_h)
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), gp)
    n1 = 72 * p.hopf_n**3
    n = p.n_rotations
    k, V, M, C, r = ctx.debug(pb, n)
    ctx.destroy_target(t)
    assert r.status == 0 and r.rot_index == argmin_cost(C)
    P = oracle_params(p, gp, p.grid_cap)
    dg = oracle.dist_grid(p.Y, 128, P.grid_cap, threads=THREADS)
    rng = np.random.default_rng(5)
    # first pass: sampled rotations, the max-V one and the first-pass winner
    idx1 = sorted(set(rng.choice(n1, size=12, replace=False).tolist()) | {int(np.argmax(V[:n1])),
                                                                           argmin_cost(C[:n1])})
    R1 = [oracle.hopf_rotation(p.hopf_n, i) for i in idx1]
    rep = check_parallel(p.X, p.Y, R1, P, k, V, M, C, idx1, dist_grid=dg)
    print("parity robot_like first pass:", rep.summary())
    assert rep.ok(), rep.summary()
    # second pass: the GPU's centres are the refine_top_k best first-pass
    # rotations by (cost, index); the oracle rebuilds their Euler boxes in FP64
    B = (2 * p.refine_K + 1) ** 3
    c1 = np.where(np.isfinite(C[:n1]), C[:n1], np.inf)
    centres = np.lexsort((np.arange(n1), c1))[: p.refine_top_k]
    boxes = {}
    idx2 = sorted(set((n1 + rng.choice(p.refine_top_k * B, size=20, replace=False)).tolist())
                  | ({r.rot_index} if r.rot_index >= n1 else set()))
    R2 = []
    for gi in idx2:
        c, local = divmod(gi - n1, B)
        if c not in boxes:
            boxes[c] = oracle.euler_box(oracle.hopf_rotation(p.hopf_n, int(centres[c])), p.refine_K,
                                        float(gp.refine_delta_r))
        R2.append(boxes[c][local])
    rep2 = check_parallel(p.X, p.Y, R2, P, k, V, M, C, idx2, dist_grid=dg)
    print("parity robot_like second pass:", rep2.summary())
    assert rep2.ok(), rep2.summary()
    # the winner is no worse than any first-pass rotation (the second pass only adds candidates)
    assert r.cost <= np.nanmin(C[:n1]) + 1e-7
