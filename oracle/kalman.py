"""Constant-velocity Kalman filter on the frame estimates, FP64 (test
infrastructure only).

The temporal filter of Sec. III-A written in its textbook matrix form: state
s = [Theta, dTheta/dt] (2d entries, joint coordinates as joint angles q),
motion s_t = F s_{t-1} + w with F = [[I, dt I], [0, I]], w ~ N(0, Q);
measurement z_t = [I 0] s_t + v, v ~ N(0, R), where z_t is the tracker's
frame estimate.  Prediction s = F s, P = F P F^T + Q; update
K = P H^T (H P H^T + R)^-1, s += K (z - H s), P = (I - K H) P.  The filtered
joint angles are clamped to their limits.  First frame: s = (z, 0),
P = blockdiag(R, diag(p_vel0)).  Q = blockdiag(diag(q_pos), diag(q_vel)) and
R = diag(r): the noise values are not printed in the paper and are inputs.
"""
from __future__ import annotations

import numpy as np

from . import q_from_qhat, qhat_from_q


class Kalman:
    def __init__(self, d: int, dt: float, q_pos, q_vel, r, p_vel0, q_lb, q_ub):
        self.d = d
        I, Z = np.eye(d), np.zeros((d, d))
        self.F = np.block([[I, dt * I], [Z, I]])
        self.H = np.hstack([I, Z])
        self.Q = np.diag(np.concatenate([np.broadcast_to(q_pos, (d,)), np.broadcast_to(q_vel, (d,))]).astype(float))
        self.R = np.diag(np.broadcast_to(r, (d,)).astype(float))
        self.p_vel0 = np.broadcast_to(p_vel0, (d,)).astype(float)
        self.q_lb, self.q_ub = np.asarray(q_lb, float), np.asarray(q_ub, float)
        self.s = None
        self.P = None

    def _joints(self):
        return [(i, i % 9 - 6) for i in range(self.d) if i % 9 >= 6]

    def to_angles(self, theta):
        """State vector with q-hat joints -> Theta with joint angles."""
        z = np.array(theta, float)
        for i, j in self._joints():
            z[i] = q_from_qhat(z[i], self.q_lb[j], self.q_ub[j])
        return z

    def to_state(self, x):
        """Filter position (joint angles) -> state vector: joints clamped, then q-hat."""
        out = np.array(x, float)
        for i, j in self._joints():
            out[i] = qhat_from_q(min(self.q_ub[j], max(self.q_lb[j], out[i])), self.q_lb[j], self.q_ub[j])
        return out

    def predict(self):
        """Prior for the next frame; returns its position in state units."""
        self.s = self.F @ self.s
        self.P = self.F @ self.P @ self.F.T + self.Q
        return self.to_state(self.s[: self.d])

    def update(self, estimate):
        """Measurement = the frame's estimate (state units); returns the filtered state."""
        z = self.to_angles(estimate)
        d = self.d
        if self.s is None:
            self.s = np.concatenate([z, np.zeros(d)])
            self.P = np.diag(np.concatenate([np.diag(self.R), self.p_vel0]))
        else:
            S = self.H @ self.P @ self.H.T + self.R
            K = self.P @ self.H.T @ np.linalg.inv(S)
            self.s = self.s + K @ (z - self.H @ self.s)
            self.P = (np.eye(2 * d) - K @ self.H) @ self.P
        return self.to_state(self.s[:d])
