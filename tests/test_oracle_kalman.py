"""Pins of the oracle's constant-velocity Kalman filter (temporal filtering,
Sec. III-A): least-squares limit, exact tracking, prediction algebra and the
joint-limit clamp."""
import numpy as np
import pytest

from oracle import q_from_qhat, qhat_from_q
from oracle.kalman import Kalman

LB, UB = [-np.pi / 2, -np.pi / 2, 0.0], [np.pi / 2, np.pi / 2, 0.8]


def test_without_process_noise_the_filter_is_the_regularised_least_squares_line():
    """Q = 0: the filter's posterior after N measurements of variance r is the
    straight line x(t) = x0 + v t minimising sum_n (z_n - x0 - v t_n)^2 / r
    + v^2 / p_vel0 (the first frame's N(0, p_vel0) velocity prior), evaluated
    at the last time: solve the 2x2 normal equations directly."""
    rng = np.random.default_rng(0)
    d, dt, N, r, pv = 6, 1 / 30, 25, 0.04, 1e4
    kf = Kalman(d, dt, 0.0, 0.0, r, pv, LB, UB)
    t = np.arange(N) * dt
    a, b = rng.normal(size=d), rng.normal(size=d)
    Z = a[None] + b[None] * t[:, None] + rng.normal(size=(N, d)) * 0.2
    for n in range(N):
        if n:
            kf.predict()
        x = kf.update(Z[n])
    A = np.array([[N / r, t.sum() / r], [t.sum() / r, (t * t).sum() / r + 1 / pv]])
    for i in range(d):
        x0, v = np.linalg.solve(A, np.array([Z[:, i].sum() / r, (t * Z[:, i]).sum() / r]))
        assert x[i] == pytest.approx(x0 + v * t[-1], rel=1e-10, abs=1e-10)
        assert kf.s[d + i] == pytest.approx(v, rel=1e-9)


def test_noise_free_constant_velocity_is_tracked_exactly():
    d, dt = 9, 0.1
    kf = Kalman(d, dt, 0.0, 0.0, 1e-6, 1e12, LB, UB)
    v = np.array([0.01, -0.02, 0.03, 1.0, -2.0, 0.5, 0.0, 0.0, 0.0])
    x0 = np.array([0.1, 0.2, 0.3, 1.0, 2.0, 100.0, 0.0, 0.0, 0.4])
    for n in range(10):
        truth = x0 + v * n * dt
        if n:
            pred = kf.predict()
            if n >= 3:
                assert np.allclose(pred[:6], truth[:6], atol=1e-9)
        kf.update(truth)
    assert np.allclose(kf.s[9:15], v[:6], atol=1e-7)


def test_prediction_algebra_and_joint_clamp():
    d, dt = 9, 0.5
    kf = Kalman(d, dt, 1e-3, 1e-2, 1e-2, 1.0, LB, UB)
    kf.update(np.array([0.0, 0.0, 0.0, 0.0, 0.0, 100.0, 0.0, 0.0, 0.7]))
    kf.s[d + 8] = 1.0  # jaw opening fast: the prediction passes its limit (0.8 rad)
    s0, P0 = kf.s.copy(), kf.P.copy()
    pred = kf.predict()
    assert np.allclose(kf.s[:d], s0[:d] + dt * s0[d:])
    F = np.block([[np.eye(d), dt * np.eye(d)], [np.zeros((d, d)), np.eye(d)]])
    assert np.allclose(kf.P, F @ P0 @ F.T + kf.Q)
    # the jaw angle q(0.7) + 0.5 ~ 1.27 rad is clamped to 0.8 before the q-hat map
    assert kf.s[8] == pytest.approx(q_from_qhat(0.7, 0.0, 0.8) + 0.5)
    assert pred[8] == pytest.approx(qhat_from_q(0.8, 0.0, 0.8))
    assert q_from_qhat(pred[8], 0.0, 0.8) == pytest.approx(0.8)
