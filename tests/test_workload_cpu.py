"""The synthetic input generators against the recipes they state (the inputs
every parity test and the bench are built from): occlusion and flip rates,
trajectory amplitudes and frequencies, population spreads, detection noise,
pose sampling bounds and the paper-style mask corruption."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_11404_gb300 import workload as wl


@pytest.fixture(scope="module")
def clean_mask():
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(3)
    while True:
        M = oracle.render(sc, wl.sample_state(rng, sc.K))
        if M.sum() > 800:
            return M


def test_corrupt_mask_occludes_tool_pixels_then_flips(clean_mask):
    M = clean_mask.astype(bool)
    n_tool = M.sum()
    for seed in range(8):
        obs = wl.corrupt_mask(clean_mask, np.random.default_rng(seed), flip_p=0.0).astype(bool)
        assert not (obs & ~M).any()  # occlusion only removes tool pixels
        hidden = (M & ~obs).sum() / n_tool
        assert 0.10 <= hidden <= 0.30 + 0.35  # stops once U[0.10, 0.30] is reached (the last ellipse may overshoot)
    flips = [(wl.corrupt_mask(clean_mask, np.random.default_rng(100 + s), occ_range=(0.0, 0.0)).astype(bool) ^ M).mean()
             for s in range(8)]
    sd = math.sqrt(0.02 * 0.98 / M.size / 8)
    assert abs(np.mean(flips) - 0.02) < 5 * sd


def test_sinusoidal_trajectory_amplitudes_and_frequencies():
    rng = np.random.default_rng(5)
    p0 = np.array([0.1, -0.2, 0.3, 1.0, -2.0, 120.0, 0.1, -0.1, 0.4])
    tr = wl.sinusoidal_trajectory(rng, p0, 600)
    dev = np.abs(tr - p0)
    assert (dev[:, [0, 1, 2, 6, 7]] <= 0.3 + 1e-12).all() and (dev[:, 3:6] <= 10.0 + 1e-12).all()
    assert (tr[:, 8] >= 0.0).all() and (tr[:, 8] <= 0.8).all()
    freqs = np.fft.rfftfreq(600, 1 / 30.0)
    for k in range(8):  # 20 s at 30 Hz: the spectral peak of each component lies in [0.5, 2] Hz
        spec = np.abs(np.fft.rfft(tr[:, k] - tr[:, k].mean()))
        assert 0.45 <= freqs[np.argmax(spec)] <= 2.05, k


def test_population_around_spread():
    rng = np.random.default_rng(7)
    c = np.array([0.1, -0.2, 0.3, 1.0, -2.0, 120.0, 0.1, -0.1, 0.4])
    P = wl.population_around(rng, c, 20000).astype(np.float64)
    sd = wl.default_scales(9)
    for k in range(8):
        assert abs(P[:, k].mean() - c[k]) < 5 * sd[k] / math.sqrt(20000)
        assert abs(P[:, k].std() / sd[k] - 1) < 0.03
    assert P[:, 8].min() >= 0.0 and P[:, 8].max() <= 0.8


def test_noisy_detections_noise_and_invalid_rate():
    rng = np.random.default_rng(9)
    tips = np.tile([[100.0, 50.0, 100.0, 50.0]], (20000, 1))  # both tips at one point: order does not matter
    det = wl.noisy_detections(tips, rng, sigma_px=2.0, p_invalid=0.1)
    assert det.shape == (20000, 5) and det.dtype == np.float32
    assert abs(det[:, 4].mean() - 0.9) < 5 * math.sqrt(0.09 / 20000)
    err = det[:, :4] - tips
    assert abs(err.mean()) < 0.02 and abs(err.std() / 2.0 - 1) < 0.02


def test_sample_state_bounds():
    from scipy.spatial.transform import Rotation
    K = wl.intrinsics("c2")
    rng = np.random.default_rng(11)
    for _ in range(500):
        x = wl.sample_state(rng, K)
        R = Rotation.from_rotvec(x[:3]).as_matrix()
        back = R @ np.array([0.0, 0.0, -1.0])  # shaft direction, tip to back end
        assert back[2] >= math.cos(math.radians(60.0)) - 1e-9
        assert 80.0 <= x[5] <= 150.0
        assert abs(K.fx * x[3] / x[5]) <= 0.3 * K.width + 1e-9 and abs(K.fy * x[4] / x[5]) <= 0.3 * K.height + 1e-9
        assert -0.6 <= x[6] <= 0.6 and -0.6 <= x[7] <= 0.6 and 0.0 <= x[8] <= 0.8


def test_paper_corrupt_mask_changes_only_near_the_boundary(clean_mask):
    from scipy import ndimage
    M = clean_mask.astype(bool)
    dist_in = ndimage.distance_transform_edt(M)
    dist_out = ndimage.distance_transform_edt(~M)
    for seed in range(8):
        obs = wl.paper_corrupt_mask(clean_mask, np.random.default_rng(seed)).astype(bool)
        changed = obs ^ M
        d = np.where(M, dist_in, dist_out)[changed]
        # morphology moves the boundary by at most 2 px (square element: up to
        # 2 sqrt(2)); blobs of radius <= 8 sit on the moved boundary
        assert d.size == 0 or d.max() <= 2 * math.sqrt(2) + 8 + 1.5
