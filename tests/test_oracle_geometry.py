"""Pins for the oracle's reparameterisation, rotations, kinematics, projection
and snapping (CPU only).  References are scipy's rotations, closed forms and
an independent composition of the chain written with scipy objects."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2603_11404_gb300 import workload as wl


# --- cosine reparameterisation (Sec. III-A.3) --------------------------------

@pytest.mark.parametrize("lb,ub", [(-math.pi / 2, math.pi / 2), (0.0, 0.8), (-1.0, 2.5)])
def test_reparam_roundtrip_endpoints_range(lb, ub):
    for q in np.linspace(lb, ub, 41):
        qh = oracle.qhat_from_q(q, lb, ub)
        assert lb - 1e-12 <= qh <= ub + 1e-12
        assert abs(oracle.q_from_qhat(qh, lb, ub) - q) < 1e-9
    assert abs(oracle.q_from_qhat(lb, lb, ub) - lb) < 1e-15
    assert abs(oracle.q_from_qhat(ub, lb, ub) - ub) < 1e-12
    rng = np.random.default_rng(0)
    P = 2 * (ub - lb)
    for qh in rng.uniform(-20, 20, 200):
        q = oracle.q_from_qhat(qh, lb, ub)
        assert lb - 1e-12 <= q <= ub + 1e-12          # any sample respects the limits
        assert abs(oracle.q_from_qhat(qh + P, lb, ub) - q) < 1e-9   # 2(ub-lb)-periodic
        assert abs(oracle.q_from_qhat(2 * lb - qh, lb, ub) - q) < 1e-9  # mirror about lb


def test_reparam_flat_at_limits_and_midpoint():
    lb, ub = 0.0, 0.8
    h = 1e-6
    d_lb = (oracle.q_from_qhat(lb + h, lb, ub) - oracle.q_from_qhat(lb - h, lb, ub)) / (2 * h)
    assert abs(d_lb) < 1e-6   # no pile-up at the bounds: the map is flat there
    mid = 0.5 * (lb + ub)
    assert abs(oracle.q_from_qhat(mid, lb, ub) - mid) < 1e-15
    d_mid = (oracle.q_from_qhat(mid + h, lb, ub) - oracle.q_from_qhat(mid - h, lb, ub)) / (2 * h)
    assert abs(d_mid - math.pi / 2) < 1e-6


# --- rotations ---------------------------------------------------------------

def test_axis_angle_matches_scipy():
    rng = np.random.default_rng(1)
    for r in list(rng.normal(size=(40, 3)) * 1.5) + [np.array([1e-9, -2e-9, 0.0]), np.zeros(3)]:
        R = oracle.rotation(wl.ROT_AXIS_ANGLE, r)
        assert np.allclose(R, Rotation.from_rotvec(r).as_matrix(), atol=1e-14)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14


def test_lookat_order_and_special_cases():
    rng = np.random.default_rng(2)
    for a, b, g in rng.uniform(-3, 3, (40, 3)):
        R = oracle.rotation(wl.ROT_LOOKAT, [a, b, g])
        ref = Rotation.from_euler("YXZ", [g, a, b]).as_matrix()   # Ry(g) Rx(a) Rz(b)
        assert np.allclose(R, ref, atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
    a = 0.7
    assert np.allclose(oracle.rotation(1, [a, 0, 0]), Rotation.from_euler("x", a).as_matrix(), atol=1e-15)
    assert np.allclose(oracle.rotation(1, [0, a, 0]), Rotation.from_euler("z", a).as_matrix(), atol=1e-15)
    assert np.allclose(oracle.rotation(1, [0, 0, a]), Rotation.from_euler("y", a).as_matrix(), atol=1e-15)
    # the order matters on non-commuting angles
    assert not np.allclose(oracle.rotation(1, [0.5, 0.6, 0.7]),
                           Rotation.from_euler("XYZ", [0.5, 0.7, 0.6]).as_matrix(), atol=1e-3)


# --- kinematics and projection ----------------------------------------------

def _scipy_chain(scene, state):
    """Camera-from-frame transforms built independently with scipy rotations."""
    q = [oracle.q_from_qhat(state[6 + i], scene.q_lb[i], scene.q_ub[i]) for i in range(3)]
    if scene.rot_param == wl.ROT_AXIS_ANGLE:
        Rc = Rotation.from_rotvec(state[:3])
    else:
        Rc = Rotation.from_euler("YXZ", [state[2], state[0], state[1]])
    frames = []
    for f in scene.frames:
        ax = {wl.AXIS_NONE: None, wl.AXIS_X: "x", wl.AXIS_Y: "y", wl.AXIS_Z: "z"}[f.axis]
        Rj = Rotation.identity() if ax is None else Rotation.from_euler(ax, f.coef * q[f.joint])
        if f.parent < 0:
            R, t = Rj, np.asarray(f.offset, float)
        else:
            Rp, tp = frames[f.parent]
            R, t = Rp * Rj, tp + Rp.apply(f.offset)
        frames.append((R, t))
    return [(Rc * R, Rc.apply(t) + state[3:6]) for R, t in frames]


@pytest.mark.parametrize("rot", [wl.ROT_AXIS_ANGLE, wl.ROT_LOOKAT])
def test_chain_and_projection_against_scipy(rot):
    sc = wl.make_scene("c1", "c1", rot_param=rot)
    rng = np.random.default_rng(3)
    verts, _, vframe = sc.flat()
    for _ in range(5):
        st = wl.sample_state(rng, sc.K, rot_param=rot)
        st[6:] = rng.uniform(-2, 2, 3)  # joints anywhere: the reparam folds them into the limits
        pr = oracle.project(sc, st)
        ref = _scipy_chain(sc, st)
        for f, (R, t) in enumerate(ref):
            assert np.allclose(pr["T"][f][:, :3], R.as_matrix(), atol=1e-12)
            assert np.allclose(pr["T"][f][:, 3], t, atol=1e-10)
        X = np.stack([ref[fr][0].apply(v.astype(np.float64)) + ref[fr][1] for v, fr in zip(verts, vframe)])
        u = sc.K.fx * X[:, 0] / X[:, 2]
        v = sc.K.fy * X[:, 1] / X[:, 2]
        assert np.allclose(pr["uv"][:, 0], u, atol=1e-9) and np.allclose(pr["uv"][:, 1], v, atol=1e-9)
        assert pr["flag"].sum() == 0


def test_identity_pose_and_depth_scaling():
    sc = wl.make_scene("c1", "c1")
    st = np.zeros(9)
    st[5] = 400.0  # shaft z in [-300, 0] -> camera depth 100..400
    pr = oracle.project(sc, st)
    verts, _, vframe = sc.flat()
    sel = vframe == 0  # rigid shaft frame: X = v + t
    v = verts[sel].astype(np.float64)
    assert np.allclose(pr["uv"][sel, 0], sc.K.fx * v[:, 0] / (v[:, 2] + 400.0), atol=1e-12)
    st2 = st.copy(); st2[5] = 800.0
    pr2 = oracle.project(sc, st2)
    assert np.allclose(pr2["uv"][sel, 0] * (v[:, 2] + 800.0), pr["uv"][sel, 0] * (v[:, 2] + 400.0), atol=1e-9)


def test_zero_joints_give_rigid_chain():
    sc = wl.make_scene("c1", "c1")
    st = np.array([0.3, -0.2, 0.1, 5.0, -3.0, 120.0, 0.0, 0.0, 0.0])  # qhat = 0 -> q = 0
    pr = oracle.project(sc, st)
    R = Rotation.from_rotvec(st[:3]).as_matrix()
    offs = {0: np.zeros(3), 1: np.zeros(3), 2: np.array([0, 0, 9.0]), 3: np.array([0, 0, 9.0]), 4: np.array([0, 0, 9.0])}
    for f in range(5):
        assert np.allclose(pr["T"][f][:, :3], R, atol=1e-14)
        assert np.allclose(pr["T"][f][:, 3], R @ offs[f] + st[3:6], atol=1e-12)


def test_snap_round_half_even_and_offset():
    class K:  # fx = 256, cx = 3.5 so that 256 cx is an integer
        fx = fy = 256.0; cx = 3.5; cy = 2.0; width = 8; height = 8; z_near = 1.0
    sc = wl.Scene(wl.instrument_frames()[:1], [wl.LinkMesh(0, np.array(
        [[2.5 / 512, 0, 0], [3.5 / 512, 0, 0], [-2.5 / 512, -1.5 / 512, 0], [0.25 / 512, 0, 0]], np.float32),
        np.array([[0, 1, 2]], np.int32))], wl.Q_LB, wl.Q_UB, K())
    pr = oracle.project(sc, np.array([0, 0, 0, 0, 0, 128.0, 0, 0, 0]))
    # 256 (u - cx) = 512 X / 128 ... = 2.5, 3.5, -2.5, 0.25 exactly
    assert list(pr["snap"][:, 0]) == [2 + 896, 4 + 896, -2 + 896, 0 + 896]
    assert pr["snap"][2, 1] == -2 + 512


def test_near_plane_and_guard_band_flags():
    sc = wl.make_scene("c1", "c1")
    st = np.zeros(9); st[5] = 150.0  # shaft reaches z = -150 < z_near
    pr = oracle.project(sc, st)
    verts, _, vframe = sc.flat()
    z = verts[:, 2] + 150.0
    assert np.array_equal(pr["flag"].astype(bool), ~(z >= 1.0))
    st[3] = 1e5  # far off-axis: outside the guard band
    pr = oracle.project(sc, st)
    assert pr["flag"][z >= 1.0].all()


def test_population_counts_match_direct_render():
    sc = wl.make_scene("c1", "c1", n_instruments=2)
    rng = np.random.default_rng(5)
    a = wl.sample_state(rng, sc.K); b = wl.sample_state(rng, sc.K)
    gt = np.concatenate([a, b])
    M = oracle.render(sc, gt)
    P = wl.population_around(rng, gt, 6)
    c = oracle.eval_population(sc, P, M, n_threads=3)
    for k in range(6):
        S = oracle.render(sc, P[k].astype(np.float64))
        s, m, I, x = oracle.counts(S, M)
        assert (c["s"][k], c["m"][k], c["I"][k], c["xor"][k]) == (s, m, I, x)
    # bi-manual union is the OR of the two arms' silhouettes
    Sa = oracle.render(wl.make_scene("c1", "c1"), a)
    Sb = oracle.render(wl.make_scene("c1", "c1"), b)
    assert np.array_equal(M, Sa | Sb)


def test_backface_cull_close_to_full_union():
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(6)
    st = wl.sample_state(rng, sc.K)
    pr = oracle.project(sc, st)
    _, tris, _ = sc.flat()
    S_all, f_all, _, _ = oracle.raster(pr["snap"], pr["flag"], tris, sc.K.width, sc.K.height, False)
    S_front, f_front, _, _ = oracle.raster(pr["snap"], pr["flag"], tris, sc.K.width, sc.K.height, True)
    assert (S_front & ~S_all).sum() == 0
    assert (S_all ^ S_front).sum() <= 0.1 * S_all.sum()   # closed meshes: front faces cover the outline
    assert f_front < 0.7 * f_all                         # about half the faces are back-facing
