"""Pins of the oracle's keypoint term (Eq. kpts_loss)."""
import numpy as np
import pytest

import oracle
from oracle import keypoints as kp
from paper_2603_11404_gb300 import workload as wl


def test_kpts_loss_closed_forms():
    p = np.array([10.0, 20.0, 40.0, 25.0])
    assert kp.kpts_loss(p, p, 1.0) == 0.0
    assert kp.kpts_loss(p[[2, 3, 0, 1]], p, 0.0) == pytest.approx(0.0)  # assignment-free
    shift = np.array([3.0, 4.0, 3.0, 4.0])  # both detections 5 px off: 5 + 5 + 5 (mean)
    assert kp.kpts_loss(p + shift, p, 0.0) == pytest.approx(15.0)
    assert kp.kpts_loss(p + shift, p, 2.0) == pytest.approx(9.0)  # each term reduced by tau
    assert kp.kpts_loss(p + shift * 0.1, p, 1.0) == 0.0  # within the threshold
    one = p.copy()
    one[0] += 6.0  # one tip 6 px off: 6 + 0 + 3 (the mean moves by half)
    assert kp.kpts_loss(one, p, 0.0) == pytest.approx(9.0)


def test_projection_equals_projecting_a_mesh_vertex_at_the_keypoint():
    """The keypoint projection and the mesh projection of a vertex placed at
    the keypoint (a separate code path through the renderer's projection)."""
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(4)
    x = wl.sample_state(rng, sc.K)
    frames, pts = (3, 4), (wl.JAW_TIP, wl.JAW_TIP)
    got = kp.project_keypoints(sc, x, frames, pts)
    for k in range(2):
        one = wl.make_scene("c1", "c1")
        one.meshes = [wl.LinkMesh(frames[k], np.array([wl.JAW_TIP], np.float32), np.zeros((0, 3), np.int32))]
        pr = oracle.project(one, x)
        assert got[0, 2 * k] == pytest.approx(pr["uv"][0, 0] + sc.K.cx, abs=1e-9)
        assert got[0, 2 * k + 1] == pytest.approx(pr["uv"][0, 1] + sc.K.cy, abs=1e-9)


def test_keypoint_term_sums_valid_instruments():
    sc = wl.make_scene("c1", "c1", n_instruments=2)
    rng = np.random.default_rng(8)
    x = np.concatenate([wl.sample_state(rng, sc.K), wl.sample_state(rng, sc.K)])
    frames, pts = (3, 4), (wl.JAW_TIP, wl.JAW_TIP)
    proj = kp.project_keypoints(sc, x, frames, pts)
    obs = np.zeros((2, 5))
    obs[:, :4] = proj + 2.0
    obs[0, 4] = 1.0
    one = kp.kpts_loss(obs[0, :4], proj[0], 0.5)
    assert kp.keypoint_term(sc, x, obs, frames, pts, 0.5, 0.1) == pytest.approx(0.1 * one)
    obs[1, 4] = 1.0
    assert kp.keypoint_term(sc, x, obs, frames, pts, 0.5, 0.1) == pytest.approx(0.2 * one)
