"""Synthetic input generators: determinism, the shapes the workloads state, and
that the planted pose maps the source onto the target."""
import numpy as np
from scipy.spatial import cKDTree

from paper_2502_00115_b300 import synth


def nn_median(p):
    d, _ = cKDTree(p.Y).query(p.X @ np.asarray(p.R_true).T + np.asarray(p.t_true))
    return float(np.median(d))


def test_modelnet_like_sizes_pose_and_determinism():
    a = synth.modelnet_like_problem(4)
    b = synth.modelnet_like_problem(4)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y)
    assert a.X.shape == (717, 3) and a.Y.shape == (1024, 3)
    assert a.X.dtype == np.float32 and a.Y.dtype == np.float32
    # unit-sphere normalised target; independent noisy samples of one surface
    assert np.linalg.norm(a.Y, axis=1).max() < 1.1
    assert nn_median(a) < 0.06
    R = np.asarray(a.R_true)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(R) - 1) < 1e-12


def test_euler_rotation_range_and_rotated_frame():
    for seed in range(5):
        p = synth.modelnet_like_problem(seed, max_euler_deg=45.0)
        q = synth.modelnet_like_problem(seed, max_euler_deg=45.0, rotated_frame=True)
        # the rotated frame keeps the relative pose's angle and the fit
        ang = lambda R: np.degrees(np.arccos(np.clip((np.trace(np.asarray(R)) - 1) / 2, -1, 1)))
        assert abs(ang(p.R_true) - ang(q.R_true)) < 1e-9
        assert abs(nn_median(p) - nn_median(q)) < 1e-5
        # three Euler angles within +-45 deg turn by at most 85.8 deg (the
        # largest over a 31^3 sweep of the angle box)
        assert ang(p.R_true) < 86.0


def test_robot_like_and_tiny_shapes():
    r = synth.robot_like_problem(0, hopf_n=2, refine_top_k=0)
    assert r.X.shape == (5000, 3) and r.Y.shape == (20000, 3)
    t = synth.tiny_problem(0)
    assert t.X.shape == (128, 3) and t.Y.shape == (256, 3)
    assert nn_median(t) < 0.02
