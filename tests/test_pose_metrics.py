"""Pose-error measures of the quality workload (Section V-A metrics), checked
against closed forms."""
import math

import numpy as np

import bench


def rz(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])


def rx(deg):
    a = math.radians(deg)
    return np.array([[1.0, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])


def test_single_axis_rotation_errors():
    # a rotation by theta about z: isotropic angle theta; of the three 'zyx'
    # Euler angles only the z one changes, so the mean absolute error is theta / 3
    e = bench.pose_errors(rz(12.0), [0.3, -0.1, 0.2], np.eye(3), np.zeros(3))
    assert abs(e["mie_r"] - 12.0) < 1e-9
    assert abs(e["mae_r"] - 4.0) < 1e-9
    assert abs(e["mie_t"] - math.sqrt(0.09 + 0.01 + 0.04)) < 1e-12
    assert abs(e["mae_t"] - 0.2) < 1e-12


def test_isotropic_error_is_frame_invariant():
    rng = np.random.default_rng(0)
    from scipy.spatial.transform import Rotation

    R = Rotation.random(random_state=1).as_matrix()
    D = rx(7.0) @ rz(-5.0)
    base = bench.pose_errors(R @ D, np.zeros(3), R, np.zeros(3))["mie_r"]
    for _ in range(3):
        Q = Rotation.random(random_state=int(rng.integers(1000))).as_matrix()
        e = bench.pose_errors(Q @ R @ D @ Q.T, np.zeros(3), Q @ R @ Q.T, np.zeros(3))["mie_r"]
        assert abs(e - base) < 1e-9
    # exact: the angle of D = Rx(7) Rz(-5) from its trace
    ang = math.degrees(math.acos((np.trace(D) - 1) / 2))
    assert abs(base - ang) < 1e-9


def test_recall_thresholds():
    errs = [dict(mie_r=0, mie_t=0, mae_r=0.5, mae_t=0.05), dict(mie_r=0, mie_t=0, mae_r=1.5, mae_t=0.05),
            dict(mie_r=0, mie_t=0, mae_r=0.5, mae_t=0.2), dict(mie_r=0, mie_t=0, mae_r=0.99, mae_t=0.099)]
    s = bench.summarise_errors(errs)
    assert s["recall"] == 0.5
    assert abs(s["mae_r"] - (0.5 + 1.5 + 0.5 + 0.99) / 4) < 1e-12
