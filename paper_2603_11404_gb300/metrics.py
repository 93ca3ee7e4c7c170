"""Pose-error metrics of Sec. IV-B, for evaluating trackers (benchmarks, tests).

Per instrument of a state (layout [r | t | q-hat], 9 entries per instrument):
* rotation: the geodesic angle between the estimated and the true rotation,
  arccos((trace(R_est^T R_true) - 1) / 2), in rad;
* translation: the Euclidean distance between the translations, in mm;
* joints: |q_est - q_true| for wrist pitch, wrist yaw and jaw, in rad of joint
  angle, with q from the state's unconstrained coordinate q-hat by the inverse
  cosine map q = lb + (ub - lb)/2 (1 - cos(pi (q-hat - lb)/(ub - lb))) of
  Sec. III-A.3.

Evaluation only: no kernel or oracle computation uses this module.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

from . import workload as wl


def rotation_matrix(r, rot_param: int = wl.ROT_AXIS_ANGLE) -> np.ndarray:
    """3x3 rotation of the state's rotation parameters (axis-angle vector or
    the look-at angles alpha, beta, gamma of Sec. III-A.3)."""
    r = np.asarray(r, np.float64)
    if rot_param == wl.ROT_LOOKAT:
        return wl.matrix_from_lookat(r)
    return Rotation.from_rotvec(r).as_matrix()


def joint_angles(qhat, q_lb, q_ub) -> np.ndarray:
    qhat, lb, ub = (np.asarray(x, np.float64) for x in (qhat, q_lb, q_ub))
    rng = np.where(ub > lb, ub - lb, 1.0)
    return np.where(ub > lb, lb + 0.5 * (ub - lb) * (1.0 - np.cos(np.pi * (qhat - lb) / rng)), lb)


def pose_errors(est, true, q_lb=wl.Q_LB, q_ub=wl.Q_UB, rot_param: int = wl.ROT_AXIS_ANGLE) -> dict:
    """Errors of one estimate against the true state, per instrument: arrays
    rot [n_inst] (rad), trans [n_inst] (mm), joints [n_inst, 3] (rad)."""
    est, true = np.asarray(est, np.float64), np.asarray(true, np.float64)
    n = est.shape[0] // 9
    rot, trans, joints = np.zeros(n), np.zeros(n), np.zeros((n, 3))
    for b in range(n):
        e, t = est[9 * b: 9 * b + 9], true[9 * b: 9 * b + 9]
        Re, Rt = rotation_matrix(e[:3], rot_param), rotation_matrix(t[:3], rot_param)
        c = (np.trace(Re.T @ Rt) - 1.0) / 2.0
        rot[b] = float(np.arccos(np.clip(c, -1.0, 1.0)))
        trans[b] = float(np.linalg.norm(e[3:6] - t[3:6]))
        joints[b] = np.abs(joint_angles(e[6:9], q_lb, q_ub) - joint_angles(t[6:9], q_lb, q_ub))
    return {"rot": rot, "trans": trans, "joints": joints}


def summarise(errors) -> dict:
    """Mean, standard error and median of a list of pose_errors results
    (pooled over frames and instruments; joints pooled over the three)."""
    rot = np.concatenate([e["rot"] for e in errors])
    trans = np.concatenate([e["trans"] for e in errors])
    joints = np.concatenate([e["joints"].reshape(-1) for e in errors])
    out = {}
    for k, v in (("rot_rad", rot), ("trans_mm", trans), ("joint_rad", joints)):
        out[k] = {"mean": float(v.mean()), "se": float(v.std(ddof=1) / np.sqrt(len(v))) if len(v) > 1 else 0.0,
                  "median": float(np.median(v))}
    return out
