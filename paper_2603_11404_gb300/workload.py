"""Seeded synthetic inputs shaped like the tracking workloads of arXiv 2603.11404.

This module only *makes data*: procedural instrument meshes, the kinematic chain
description, camera intrinsics, ground-truth states, sinusoidal trajectories and
the corruption of observed masks.  It contains none of the tracker's arithmetic
(no forward kinematics, projection, rasterisation, loss or CMA-ES); both the CUDA
path and the CPU oracle consume what it returns.

The paper's own inputs (CAD meshes of the Large Needle Driver, the synthetic
700x493 set, SurgPose and the collected 640x480 stereo set; Sec. IV) are not
available, so every input here is a seeded stand-in of the same shape:

* The instrument follows Sec. III-A: a 6-DoF end-effector pose at the wrist-pitch
  frame plus wrist pitch q1, wrist yaw q2 and jaw angle q3.  The paper gives no
  link geometry, so the mesh is procedural: a 4.2 mm-radius, 300 mm shaft, an
  8x5x10 mm wrist box and two 10 mm jaw wedges, subdivided to a target triangle
  count (about 1.5k for the 160x128 fit, about 20k for the 640x512 tracking set).
* State vectors are ``[r0, r1, r2, x, y, z, qh1, qh2, qh3]`` per instrument: a
  rotation (axis-angle, or look-at angles alpha, beta, gamma of Sec. III-A.3), a
  translation in mm and the *unconstrained* joint coordinates q-hat of the cosine
  reparameterisation (Sec. III-A.3).  Joint samples are drawn directly in q-hat.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Joint axis codes shared with include/tracker.h (TRK_AXIS_*).
AXIS_NONE, AXIS_X, AXIS_Y, AXIS_Z = 0, 1, 2, 3
# Rotation parameterisations (TRK_ROT_*).
ROT_AXIS_ANGLE, ROT_LOOKAT = 0, 1
# Loss kinds (TRK_LOSS_*).
LOSS_XOR, LOSS_ONE_MINUS_IOU, LOSS_MSE_APP = 0, 1, 2

D_PER_INSTRUMENT = 9


@dataclasses.dataclass
class Frame:
    """One kinematic frame: T = T_parent * Trans(offset) * Rot(axis, coef * q[joint])."""
    parent: int
    offset: tuple
    axis: int = AXIS_NONE
    joint: int = 0
    coef: float = 0.0


@dataclasses.dataclass
class LinkMesh:
    frame: int
    verts: np.ndarray  # float32 [n, 3], mm, in the frame's coordinates
    tris: np.ndarray   # int32 [m, 3], indices into verts


@dataclasses.dataclass
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 1.0


@dataclasses.dataclass
class Scene:
    frames: List[Frame]
    meshes: List[LinkMesh]
    q_lb: np.ndarray
    q_ub: np.ndarray
    K: Intrinsics
    n_instruments: int = 1
    rot_param: int = ROT_AXIS_ANGLE

    @property
    def d(self) -> int:
        return D_PER_INSTRUMENT * self.n_instruments

    @property
    def n_tris(self) -> int:
        return int(sum(m.tris.shape[0] for m in self.meshes))

    @property
    def n_verts(self) -> int:
        return int(sum(m.verts.shape[0] for m in self.meshes))

    def flat(self):
        """Concatenated vertex/triangle arrays plus the frame id of every vertex."""
        vs, ts, fr = [], [], []
        base = 0
        for m in self.meshes:
            vs.append(m.verts)
            ts.append(m.tris + base)
            fr.append(np.full(m.verts.shape[0], m.frame, np.int32))
            base += m.verts.shape[0]
        return (np.ascontiguousarray(np.concatenate(vs).astype(np.float32)),
                np.ascontiguousarray(np.concatenate(ts).astype(np.int32)),
                np.ascontiguousarray(np.concatenate(fr).astype(np.int32)))


# --------------------------------------------------------------------------
# Procedural meshes
# --------------------------------------------------------------------------

class _MeshBuilder:
    """Collects triangles of a convex solid, merging equal vertices and winding
    every triangle counter-clockwise seen from outside (normal away from the
    solid's centroid)."""

    def __init__(self, centroid):
        self.centroid = np.asarray(centroid, np.float64)
        self.index = {}
        self.verts = []
        self.tris = []

    def vid(self, p):
        key = tuple(np.round(np.asarray(p, np.float64), 6))
        if key not in self.index:
            self.index[key] = len(self.verts)
            self.verts.append(key)
        return self.index[key]

    def tri(self, a, b, c):
        pa, pb, pc = (np.asarray(x, np.float64) for x in (a, b, c))
        n = np.cross(pb - pa, pc - pa)
        if np.dot(n, n) == 0.0:
            return
        if np.dot(n, (pa + pb + pc) / 3.0 - self.centroid) < 0.0:
            pb, pc = pc, pb
        self.tris.append((self.vid(pa), self.vid(pb), self.vid(pc)))

    def quad_grid(self, p0, e1, e2, n1, n2):
        p0, e1, e2 = (np.asarray(x, np.float64) for x in (p0, e1, e2))
        P = lambda i, j: p0 + e1 * (i / n1) + e2 * (j / n2)
        for i in range(n1):
            for j in range(n2):
                self.tri(P(i, j), P(i + 1, j), P(i + 1, j + 1))
                self.tri(P(i, j), P(i + 1, j + 1), P(i, j + 1))

    def tri_lattice(self, a, b, c, n):
        a, b, c = (np.asarray(x, np.float64) for x in (a, b, c))
        P = lambda i, j: a + (b - a) * (i / n) + (c - a) * (j / n)
        for i in range(n):
            for j in range(n - i):
                self.tri(P(i, j), P(i + 1, j), P(i, j + 1))
                if i + j + 1 < n:
                    self.tri(P(i + 1, j), P(i + 1, j + 1), P(i, j + 1))

    def mesh(self, frame):
        return LinkMesh(frame, np.asarray(self.verts, np.float32),
                        np.asarray(self.tris, np.int32))


def shaft_mesh(frame=0, radius=4.2, length=300.0, segments=32, rings=20, cap_rings=1):
    """Closed cylinder along z in [-length, 0]."""
    b = _MeshBuilder((0.0, 0.0, -length / 2))
    ang = [2 * math.pi * s / segments for s in range(segments + 1)]
    ring = lambda s, z, r=radius: (r * math.cos(ang[s % segments]), r * math.sin(ang[s % segments]), z)
    for k in range(rings):
        z0 = -length + length * k / rings
        z1 = -length + length * (k + 1) / rings
        for s in range(segments):
            b.tri(ring(s, z0), ring(s + 1, z0), ring(s + 1, z1))
            b.tri(ring(s, z0), ring(s + 1, z1), ring(s, z1))
    for z in (-length, 0.0):
        for c in range(cap_rings):
            r0 = radius * c / cap_rings
            r1 = radius * (c + 1) / cap_rings
            for s in range(segments):
                if c == 0:
                    b.tri((0.0, 0.0, z), ring(s, z, r1), ring(s + 1, z, r1))
                else:
                    b.tri(ring(s, z, r0), ring(s, z, r1), ring(s + 1, z, r1))
                    b.tri(ring(s, z, r0), ring(s + 1, z, r1), ring(s + 1, z, r0))
    return b.mesh(frame)


def box_mesh(frame=1, sx=8.0, sy=5.0, sz=10.0, z0=0.0, div=(2, 2, 2)):
    """Axis-aligned box x in [-sx/2, sx/2], y in [-sy/2, sy/2], z in [z0, z0+sz]."""
    nx, ny, nz = div
    b = _MeshBuilder((0.0, 0.0, z0 + sz / 2))
    x0, y0 = -sx / 2, -sy / 2
    for zc in (z0, z0 + sz):
        b.quad_grid((x0, y0, zc), (sx, 0, 0), (0, sy, 0), nx, ny)
    for yc in (y0, y0 + sy):
        b.quad_grid((x0, yc, z0), (sx, 0, 0), (0, 0, sz), nx, nz)
    for xc in (x0, x0 + sx):
        b.quad_grid((xc, y0, z0), (0, sy, 0), (0, 0, sz), ny, nz)
    return b.mesh(frame)


def jaw_mesh(frame, side, length=10.0, base=2.5, width=4.0, div=3, ydiv=2):
    """Triangular prism (a wedge): cross-section (0,0)-(side*base,0)-(0,length) in
    the x-z plane, extruded over y in [-width/2, width/2]."""
    A = np.array([0.0, 0.0]); B = np.array([side * base, 0.0]); C = np.array([0.0, length])
    cen2 = (A + B + C) / 3
    b = _MeshBuilder((cen2[0], 0.0, cen2[1]))
    P = lambda p, y: (p[0], y, p[1])
    for y in (-width / 2, width / 2):
        b.tri_lattice(P(A, y), P(B, y), P(C, y), div)
    for p, q in ((A, B), (B, C), (C, A)):
        b.quad_grid(P(p, -width / 2), (q[0] - p[0], 0.0, q[1] - p[1]), (0.0, width, 0.0), div, ydiv)
    return b.mesh(frame)


def instrument_frames():
    """Kinematic chain of the wrist (frames in the end-effector frame E).

    E sits on the wrist-pitch axis (Sec. III-A: the end-effector frame is the
    wrist pitch frame); z runs along the shaft towards the tip, the pitch axis
    is x.  0 shaft (fixed), 1 wrist Rx(q1), 2 yaw Trans(0,0,9) Ry(q2),
    3/4 jaws Ry(+-q3/2)."""
    return [
        Frame(-1, (0.0, 0.0, 0.0)),
        Frame(-1, (0.0, 0.0, 0.0), AXIS_X, 0, 1.0),
        Frame(1, (0.0, 0.0, 9.0), AXIS_Y, 1, 1.0),
        Frame(2, (0.0, 0.0, 0.0), AXIS_Y, 2, 0.5),
        Frame(2, (0.0, 0.0, 0.0), AXIS_Y, 2, -0.5),
    ]


# Jaw tips in their frames (used by keypoint-style tests).
JAW_TIP = np.array([0.0, 0.0, 10.0])
Q_LB = np.array([-math.pi / 2, -math.pi / 2, 0.0])
Q_UB = np.array([math.pi / 2, math.pi / 2, 0.8])


def instrument_meshes(size: str = "c1"):
    """Preset subdivisions: 'c1' ~1.5k triangles, 'c2' ~20k triangles, or an
    integer-like string giving an approximate total."""
    if size == "c1":
        return [shaft_mesh(rings=20, cap_rings=1), box_mesh(div=(2, 2, 2)),
                jaw_mesh(3, +1, div=3, ydiv=2), jaw_mesh(4, -1, div=3, ydiv=2)]
    if size == "c2":
        return [shaft_mesh(rings=290, cap_rings=2), box_mesh(div=(8, 5, 10)),
                jaw_mesh(3, +1, div=8, ydiv=4), jaw_mesh(4, -1, div=8, ydiv=4)]
    target = int(size)
    # box 188 + jaws 2x80 + two 2-ring caps 128 = 476 triangles besides the shaft wall
    rings = max(2, int(round((target - 476) / 64)))
    return [shaft_mesh(rings=rings, cap_rings=2), box_mesh(div=(4, 3, 5)),
            jaw_mesh(3, +1, div=4, ydiv=2), jaw_mesh(4, -1, div=4, ydiv=2)]


def intrinsics(name: str) -> Intrinsics:
    if name == "c1":
        return Intrinsics(200.0, 200.0, 80.0, 64.0, 160, 128)
    if name == "c2":
        return Intrinsics(800.0, 800.0, 320.0, 256.0, 640, 512)
    raise ValueError(name)


def make_scene(mesh: str = "c1", cam: str = "c1", n_instruments: int = 1,
               rot_param: int = ROT_AXIS_ANGLE, K: Intrinsics | None = None) -> Scene:
    return Scene(instrument_frames(), instrument_meshes(mesh), Q_LB.copy(), Q_UB.copy(),
                 K if K is not None else intrinsics(cam), n_instruments, rot_param)


# --------------------------------------------------------------------------
# Ground-truth states and trajectories
# --------------------------------------------------------------------------

def _rotvec_from_matrix(R: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    return Rotation.from_matrix(R).as_rotvec()


def sample_state(rng: np.random.Generator, K: Intrinsics, z_range=(80.0, 150.0),
                 max_tilt_deg=60.0, central=0.6, rot_param=ROT_AXIS_ANGLE) -> np.ndarray:
    """One 9-vector: shaft direction (tip to back end) within max_tilt of +z_cam,
    uniform roll, E origin at depth z ~ U[z_range] placed so that it lies in the
    central fraction of the image, q-hat1,2 ~ U[-0.6, 0.6], q-hat3 ~ U[0, 0.8]."""
    cos_max = math.cos(math.radians(max_tilt_deg))
    cz = rng.uniform(cos_max, 1.0)
    phi = rng.uniform(0, 2 * math.pi)
    sz = math.sqrt(max(0.0, 1 - cz * cz))
    back = np.array([sz * math.cos(phi), sz * math.sin(phi), cz])  # R @ (0,0,-1)
    ez = -back
    tmp = np.array([1.0, 0.0, 0.0]) if abs(ez[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    ex = np.cross(tmp, ez); ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    roll = rng.uniform(0, 2 * math.pi)
    c, s = math.cos(roll), math.sin(roll)
    ex, ey = c * ex + s * ey, -s * ex + c * ey
    R = np.stack([ex, ey, ez], axis=1)
    z = rng.uniform(*z_range)
    x = rng.uniform(-1, 1) * central * 0.5 * K.width / K.fx * z
    y = rng.uniform(-1, 1) * central * 0.5 * K.height / K.fy * z
    if rot_param == ROT_AXIS_ANGLE:
        r = _rotvec_from_matrix(R)
    else:
        from scipy.spatial.transform import Rotation
        # R = Ry(gamma) Rx(alpha) Rz(beta): intrinsic y-x-z Euler angles.
        gamma, alpha, beta = Rotation.from_matrix(R).as_euler("YXZ")
        r = np.array([alpha, beta, gamma])
    qh = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(0.0, 0.8)])
    return np.concatenate([r, [x, y, z], qh])


def sinusoidal_trajectory(rng: np.random.Generator, p0: np.ndarray, n_frames: int,
                          fps: float = 30.0, amp_mm: float = 10.0, amp_rad: float = 0.3,
                          f_range=(0.5, 2.0), jaw_range=(0.0, 0.8)) -> np.ndarray:
    """[n_frames, 9] states: every component p0 + A sin(2 pi f t + phi) with
    f ~ U[f_range], phi ~ U[0, 2 pi); A = amp_mm for translations and amp_rad for
    rotations and joints; the jaw coordinate is clamped to jaw_range."""
    d = p0.shape[0]
    f = rng.uniform(*f_range, size=d)
    ph = rng.uniform(0, 2 * math.pi, size=d)
    A = np.full(d, amp_rad)
    for b in range(d // D_PER_INSTRUMENT):
        A[b * 9 + 3: b * 9 + 6] = amp_mm
    t = np.arange(n_frames)[:, None] / fps
    traj = p0[None, :] + A[None, :] * np.sin(2 * math.pi * f[None, :] * t + ph[None, :])
    for b in range(d // D_PER_INSTRUMENT):
        traj[:, b * 9 + 8] = np.clip(traj[:, b * 9 + 8], *jaw_range)
    return traj


def corrupt_mask(mask: np.ndarray, rng: np.random.Generator, flip_p: float = 0.02,
                 occ_range=(0.10, 0.30), max_ellipses: int = 64) -> np.ndarray:
    """Observed mask = clean mask with seeded occluding ellipses set to background
    until the occluded fraction of tool pixels reaches U[occ_range], then iid
    Bernoulli(flip_p) pixel flips over the whole image."""
    m = mask.astype(bool).copy()
    H, W = m.shape
    tool = np.argwhere(m)
    n_tool = tool.shape[0]
    if n_tool > 0:
        target = rng.uniform(*occ_range)
        occluded = np.zeros_like(m)
        tool_mask = mask.astype(bool)
        n_occ = 0
        scale = max(4.0, math.sqrt(n_tool) / 4)
        for _ in range(max_ellipses):
            if n_occ >= target * n_tool:
                break
            ci, cj = tool[rng.integers(n_tool)]
            a, b = rng.uniform(0.3, 1.0, size=2) * scale
            th = rng.uniform(0, math.pi)
            c, s = math.cos(th), math.sin(th)
            r = int(math.ceil(max(a, b))) + 1
            i0, i1, j0, j1 = max(0, ci - r), min(H, ci + r + 1), max(0, cj - r), min(W, cj + r + 1)
            ii, jj = np.mgrid[i0:i1, j0:j1]
            dx, dy = jj - cj, ii - ci
            u = (c * dx + s * dy) / a
            v = (-s * dx + c * dy) / b
            win = occluded[i0:i1, j0:j1]
            before = int((win & tool_mask[i0:i1, j0:j1]).sum())
            win |= (u * u + v * v) <= 1.0
            n_occ += int((win & tool_mask[i0:i1, j0:j1]).sum()) - before
        m &= ~occluded
    flips = rng.random((H, W)) < flip_p
    return (m ^ flips).astype(np.uint8)


def population_around(rng: np.random.Generator, center: np.ndarray, lam: int,
                      sigma_rad: float = 0.05, sigma_mm: float = 2.0) -> np.ndarray:
    """lam states drawn N(center, diag(sigma)^2) with sigma_rad on rotations and
    joints and sigma_mm on translations; the jaw coordinate stays in [0, 0.8]."""
    d = center.shape[0]
    sd = np.full(d, sigma_rad)
    for b in range(d // D_PER_INSTRUMENT):
        sd[b * 9 + 3: b * 9 + 6] = sigma_mm
    P = center[None, :] + rng.standard_normal((lam, d)) * sd[None, :]
    for b in range(d // D_PER_INSTRUMENT):
        P[:, b * 9 + 8] = np.clip(P[:, b * 9 + 8], 0.0, 0.8)
    return P.astype(np.float32)


def default_scales(d: int) -> np.ndarray:
    """Normalisation of the search space: 0.05 rad for rotations and joints, 2 mm
    for translations (the initial spread of the 160x128 fit)."""
    s = np.full(d, 0.05)
    for b in range(d // D_PER_INSTRUMENT):
        s[b * 9 + 3: b * 9 + 6] = 2.0
    return s


def noisy_detections(tips: np.ndarray, rng: np.random.Generator, sigma_px: float = 2.0,
                     p_invalid: float = 0.1) -> np.ndarray:
    """Synthetic keypoint detections from projected true keypoints tips
    [n_inst, 4] (u1, v1, u2, v2): iid N(0, sigma_px^2) noise per coordinate,
    the two tips listed in random order, and with probability p_invalid the
    detection is marked invalid (not exactly two keypoints found).  Returns
    [n_inst, 5] float32 (x1, y1, x2, y2, valid)."""
    tips = np.asarray(tips, np.float64)
    out = np.zeros((tips.shape[0], 5), np.float32)
    for b in range(tips.shape[0]):
        t = tips[b].reshape(2, 2) + rng.normal(size=(2, 2)) * sigma_px
        if rng.random() < 0.5:
            t = t[::-1]
        out[b, :4] = t.reshape(-1)
        out[b, 4] = 0.0 if rng.random() < p_invalid else 1.0
    return out


# --------------------------------------------------------------------------
# Paper-style synthetic workload (the synthetic set of Sec. IV: 700x493
# frames, smooth random motion, mask corruption by morphology and blobs)
# --------------------------------------------------------------------------
def paper_intrinsics() -> Intrinsics:
    return Intrinsics(700.0, 700.0, 350.0, 246.5, 700, 493)


def lookat_from_matrix(R: np.ndarray) -> np.ndarray:
    """Angles (alpha, beta, gamma) with R = Ry(gamma) Rx(alpha) Rz(beta)."""
    alpha = math.atan2(-R[1, 2], math.hypot(R[0, 2], R[2, 2]))
    gamma = math.atan2(R[0, 2], R[2, 2])
    beta = math.atan2(R[1, 0], R[1, 1])
    return np.array([alpha, beta, gamma])


def matrix_from_lookat(a: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    return (Rotation.from_euler("y", a[2]) * Rotation.from_euler("x", a[0]) * Rotation.from_euler("z", a[1])).as_matrix()


def state_lookat_to_axis_angle(x: np.ndarray) -> np.ndarray:
    """Same pose with the rotation as an axis-angle vector (per instrument)."""
    out = np.array(x, np.float64)
    for b in range(len(out) // D_PER_INSTRUMENT):
        out[9 * b: 9 * b + 3] = _rotvec_from_matrix(matrix_from_lookat(out[9 * b: 9 * b + 3]))
    return out


def paper_trajectory(rng: np.random.Generator, p0: np.ndarray, n_frames: int, fps: float = 30.0,
                     seg_s: float = 1.0, amp_mm: float = 10.0, amp_rad: float = 0.3, ou_theta: float = 2.0,
                     ou_sigma: float = 0.05, smooth: float = 0.3) -> np.ndarray:
    """[n_frames, d] states: cubic Hermite spline through random waypoints
    (every seg_s seconds, offsets U[-amp, amp] around p0, Catmull-Rom
    tangents), plus Ornstein-Uhlenbeck noise (rate ou_theta, scale ou_sigma x
    amp), low-pass filtered by exponential smoothing (factor smooth); jaw
    coordinates clamped to [0, 0.8]."""
    d = p0.shape[0]
    A = np.full(d, amp_rad)
    for b in range(d // D_PER_INSTRUMENT):
        A[b * 9 + 3: b * 9 + 6] = amp_mm
    n_seg = int(math.ceil(n_frames / (seg_s * fps))) + 3
    W = p0[None, :] + rng.uniform(-1, 1, size=(n_seg, d)) * A[None, :]
    T = np.zeros_like(W)
    T[1:-1] = 0.5 * (W[2:] - W[:-2])
    out = np.zeros((n_frames, d))
    ou = np.zeros(d)
    dt = 1.0 / fps
    y = None
    for f in range(n_frames):
        u = f / (seg_s * fps)
        k = int(u) + 1
        t = u - int(u)
        h00, h10, h01, h11 = 2 * t**3 - 3 * t**2 + 1, t**3 - 2 * t**2 + t, -2 * t**3 + 3 * t**2, t**3 - t**2
        x = h00 * W[k] + h10 * T[k] + h01 * W[k + 1] + h11 * T[k + 1]
        ou += -ou_theta * ou * dt + ou_sigma * A * math.sqrt(dt) * rng.normal(size=d)
        x = x + ou
        y = x if y is None else smooth * x + (1 - smooth) * y
        out[f] = y
    for b in range(d // D_PER_INSTRUMENT):
        out[:, b * 9 + 8] = np.clip(out[:, b * 9 + 8], 0.0, 0.8)
    return out


def paper_corrupt_mask(mask: np.ndarray, rng: np.random.Generator, max_radius: int = 2, n_blobs: int = 6,
                       blob_r=(2.0, 8.0), flip_p: float = 0.0) -> np.ndarray:
    """Observed mask = clean mask dilated or eroded by a random radius
    (0..max_radius px, square structuring element), then n_blobs disks centred
    on random boundary pixels, each added or removed with equal odds."""
    from scipy import ndimage
    m = mask.astype(bool)
    r = int(rng.integers(0, max_radius + 1))
    if r > 0:
        st = np.ones((2 * r + 1, 2 * r + 1), bool)
        m = ndimage.binary_dilation(m, st) if rng.random() < 0.5 else ndimage.binary_erosion(m, st)
    edge = m ^ ndimage.binary_erosion(m)
    pts = np.argwhere(edge)
    H, W = m.shape
    for _ in range(n_blobs if len(pts) else 0):
        ci, cj = pts[rng.integers(len(pts))]
        rad = rng.uniform(*blob_r)
        i0, i1 = max(0, int(ci - rad)), min(H, int(ci + rad) + 1)
        j0, j1 = max(0, int(cj - rad)), min(W, int(cj + rad) + 1)
        ii, jj = np.mgrid[i0:i1, j0:j1]
        disk = (ii - ci) ** 2 + (jj - cj) ** 2 <= rad * rad
        if rng.random() < 0.5:
            m[i0:i1, j0:j1] |= disk
        else:
            m[i0:i1, j0:j1] &= ~disk
    if flip_p > 0:
        m ^= rng.random(m.shape) < flip_p
    return m.astype(np.uint8)
