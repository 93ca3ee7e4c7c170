"""Keypoint term of the objective, FP64 (test infrastructure only).

Eq. (kpts_loss): with detected keypoints t^r_1, t^r_2 and the candidate's
projected keypoints t^p_1, t^p_2 (px),
  L_kpts = min over the two assignments sigma of sum_i (|t^r_i - t^p_sigma(i)| - tau)_+
           + (|t^r_mean - t^p_mean| - tau)_+,
evaluated only when exactly two keypoints were detected; the objective adds
lambda_kpts * L_kpts per instrument (Sec. III-B for two instruments).  The
keypoints are points fixed in kinematic frames (the jaw tips), projected with
the oracle's own frame transforms and pinhole camera.
"""
from __future__ import annotations

import numpy as np

from . import project


def project_keypoints(scene, state, frames, points):
    """[n_inst, 4] = (u1, v1, u2, v2) image coordinates of the two keypoints."""
    K = scene.K
    out = np.zeros((scene.n_instruments, 4))
    for b in range(scene.n_instruments):
        T = project(scene, np.asarray(state, np.float64)[9 * b: 9 * b + 9])["T"]
        for k in range(2):
            X = T[frames[k]] @ np.append(np.asarray(points[k], np.float64), 1.0)
            out[b, 2 * k] = K.fx * X[0] / X[2] + K.cx
            out[b, 2 * k + 1] = K.fy * X[1] / X[2] + K.cy
    return out


def kpts_loss(det, proj, tau: float) -> float:
    """L_kpts of one instrument: det, proj = (x1, y1, x2, y2)."""
    r = np.asarray(det, np.float64).reshape(2, 2)
    p = np.asarray(proj, np.float64).reshape(2, 2)
    pos = lambda x: max(0.0, x)
    same = pos(np.linalg.norm(r[0] - p[0]) - tau) + pos(np.linalg.norm(r[1] - p[1]) - tau)
    swap = pos(np.linalg.norm(r[0] - p[1]) - tau) + pos(np.linalg.norm(r[1] - p[0]) - tau)
    return min(same, swap) + pos(np.linalg.norm(r.mean(axis=0) - p.mean(axis=0)) - tau)


def keypoint_term(scene, state, obs, frames, points, tau: float, lambda_kpts: float) -> float:
    """lambda_kpts * sum of L_kpts over the instruments whose detection is valid;
    obs [n_inst, 5] = (x1, y1, x2, y2, valid)."""
    proj = project_keypoints(scene, state, frames, points)
    total = 0.0
    for b in range(scene.n_instruments):
        if obs[b][4] != 0:
            total += kpts_loss(obs[b][:4], proj[b], tau)
    return lambda_kpts * total
