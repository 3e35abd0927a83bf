"""Writes the stored oracle values of the full ModelNet-shaped problem.

    python tests/golden/make_modelnet_like_golden.py [--threads T]

Calls only the FP64 oracle (oracle/, Algorithm 2 of arXiv 2502.00115) on the
seeded synthetic inputs of synth.modelnet_like_problem(0): 717 source and
1,024 target points, the N_side 16 Hopf grid (294,912 rotations), epsilon =
delta_t = 0.04, box +-0.9, truncated L2 with tau = 0.05 on the 128^3 distance
grid capped at 0.1, every rotation a candidate. The parameters are the FP32
values the CUDA path receives, widened to FP64. Per rotation it stores the
mode's lattice index k* (relative to the box corner), its frequency V, the
inlier count M (Eq. 3), the grid cost, and the oracle's boundary counts
(pairs within 1e-5 of a voxel face, points within 1e-5 of epsilon) that
excuse an FP32 decision; plus the best rotation and SHA-256 digests of the
inputs, so a changed generator is detected instead of compared. The oracle's
threaded fan-out over rotations runs the same per-rotation arithmetic as its
single-threaded path.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2502_00115_b300 import synth  # noqa: E402  (seeded inputs only)

OUT = os.path.join(HERE, "modelnet_like_nside16_seed0.npz")


def f32(v):
    return float(np.float32(v))


def params(p):
    return oracle.make_params(metric="trunc_l2", epsilon=f32(p.epsilon), delta_t=f32(p.delta_t), tau=f32(p.tau),
                              huber_h=f32(p.huber_h), p=1.0, t_center=[f32(v) for v in p.t_center],
                              t_half=[f32(v) for v in p.t_half], nn_mode="grid", grid_res=128,
                              grid_cap=f32(2 * p.tau))


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float32).tobytes()).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    p = synth.modelnet_like_problem(0)
    P = params(p)
    grid = oracle.hopf_grid(p.hopf_n)
    lo, hi = oracle.lattice_box(P.t_center[:], P.t_half[:], P.delta_t)
    t0 = time.time()
    ref = oracle.register(p.X, p.Y, grid, P, threads=a.threads)
    dt = time.time() - t0
    k_rel = ref.k - np.asarray(lo)[None, :]
    assert k_rel.min() >= 0 and k_rel.max() < 256
    assert ref.V.max() < 65536 and ref.M.max() < 65536
    np.savez_compressed(
        OUT, x_sha256=digest(p.X), y_sha256=digest(p.Y), lo=np.asarray(lo, dtype=np.int32),
        k_rel=k_rel.astype(np.uint8), V=ref.V.astype(np.uint16), M=ref.M.astype(np.uint16),
        cost=ref.costs.astype(np.float32), n_boundary_pairs=np.minimum(ref.n_boundary_pairs, 65535).astype(np.uint16),
        n_boundary_points=np.minimum(ref.n_boundary_points, 65535).astype(np.uint16),
        best=np.int64(ref.rot_index), best_cost=np.float64(ref.cost), status=np.int32(ref.status))
    print(f"wrote {OUT}: {len(grid)} rotations in {dt:.0f} s on {a.threads} threads, best {ref.rot_index} "
          f"cost {ref.cost:.6g}, boundary pairs {int(ref.n_boundary_pairs.sum())}, "
          f"points {int(ref.n_boundary_points.sum())}")


if __name__ == "__main__":
    main()
