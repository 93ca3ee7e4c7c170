"""CPU oracle for arXiv 2603.11404's silhouette fitness and CMA-ES tracker.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
executes anything in this package; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` do.  It shares no code with the CUDA
sources: the renderer is plain C in ``oracle.c`` (FP64 geometry, exact int64
edge functions), the CMA-ES, random numbers and tracker are plain numpy in
``cmaes.py``, ``philox.py`` and ``tracker.py``, and the soft (differentiable)
silhouette loss with its gradient is plain numpy in ``soft.py``.

Scenes are duck-typed: any object with ``frames`` (parent, offset, axis, joint,
coef), ``meshes`` (frame, verts, tris), ``q_lb``, ``q_ub``, ``K`` (fx, fy, cx,
cy, width, height, z_near), ``n_instruments`` and ``rot_param``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

GUARD_PX = float(2 ** 14)  # guard band on |u - cx|, |v - cy| in px


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_q_from_qhat.restype = C.c_double
            L.orc_q_from_qhat.argtypes = [C.c_double] * 3
            L.orc_qhat_from_q.restype = C.c_double
            L.orc_qhat_from_q.argtypes = [C.c_double] * 3
            L.orc_rotation.argtypes = [C.c_int, P, P]
            L.orc_raster.restype = C.c_int64
            L.orc_raster.argtypes = [C.c_int, P, C.c_int, P, P, C.c_int, C.c_int, C.c_int, P, P, P]
            L.orc_counts.argtypes = [C.c_int, C.c_int, P, P, P]
            L.orc_eval_population.restype = C.c_int
            L.orc_eval_population.argtypes = (
                [C.c_int, P, P, P, P, P, P, P, C.c_int, C.c_int, C.c_int, P, C.c_int, P, P, C.c_int, P]
                + [C.c_double] * 6 + [C.c_int, C.c_int, C.c_int, P, P, C.c_int])
            L.orc_project_state.restype = C.c_int
            L.orc_project_state.argtypes = (
                [C.c_int, P, P, P, P, P, P, P, C.c_int, P, C.c_int, P, P] + [C.c_double] * 6
                + [P, P, P, P])
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Chain:
    """Flat arrays of a scene's kinematic chain, kept alive for ctypes calls."""

    def __init__(self, scene):
        fr = scene.frames
        self.n = len(fr)
        self.parent = np.array([f.parent for f in fr], np.int32)
        self.offset = np.array([f.offset for f in fr], np.float64).reshape(-1)
        self.axis = np.array([f.axis for f in fr], np.int32)
        self.joint = np.array([f.joint for f in fr], np.int32)
        self.coef = np.array([f.coef for f in fr], np.float64)
        self.q_lb = np.ascontiguousarray(scene.q_lb, np.float64)
        self.q_ub = np.ascontiguousarray(scene.q_ub, np.float64)
        self.rot = int(scene.rot_param)

    def args(self):
        return [self.n, _p(self.parent), _p(self.offset), _p(self.axis), _p(self.joint),
                _p(self.coef), _p(self.q_lb), _p(self.q_ub), self.rot]


def _flat_mesh(scene):
    vs, ts, fr, base = [], [], [], 0
    for m in scene.meshes:
        vs.append(np.asarray(m.verts, np.float32))
        ts.append(np.asarray(m.tris, np.int32) + base)
        fr.append(np.full(len(m.verts), m.frame, np.int32))
        base += len(m.verts)
    return (np.ascontiguousarray(np.concatenate(vs)), np.ascontiguousarray(np.concatenate(ts)),
            np.ascontiguousarray(np.concatenate(fr)))


def q_from_qhat(qh, lb, ub):
    return lib().orc_q_from_qhat(float(qh), float(lb), float(ub))


def qhat_from_q(q, lb, ub):
    return lib().orc_qhat_from_q(float(q), float(lb), float(ub))


def rotation(rot_param: int, r) -> np.ndarray:
    r = np.ascontiguousarray(r, np.float64)
    R = np.zeros(9)
    lib().orc_rotation(int(rot_param), _p(r), _p(R))
    return R.reshape(3, 3)


def project(scene, state, guard: float = GUARD_PX):
    """Project one instrument's vertices for a 9-vector state.  Returns a dict with
    uv [V,2] (px offsets from the principal point), snap [V,2] int64 (1/256 px),
    flag [V] uint8 and T [n_frames,3,4] camera-from-frame transforms."""
    ch = _Chain(scene)
    verts, _, vframe = _flat_mesh(scene)
    K = scene.K
    state = np.ascontiguousarray(state, np.float64)
    nv = verts.shape[0]
    uv = np.zeros((nv, 2)); snap = np.zeros((nv, 2), np.int64); flag = np.zeros(nv, np.uint8)
    T = np.zeros((ch.n, 12))
    lib().orc_project_state(*ch.args(), _p(state), nv, _p(verts), _p(vframe), K.fx, K.fy, K.cx,
                            K.cy, K.z_near, guard, _p(uv), _p(snap), _p(flag), _p(T))
    return {"uv": uv, "snap": snap, "flag": flag, "T": T.reshape(-1, 3, 4)}


def raster(snap, flag, tris, W: int, H: int, cull_back: bool = False):
    """Union silhouette of triangles over snapped vertices.  Returns (S [H,W]
    uint8, frags, culled, bbox_px)."""
    snap = np.ascontiguousarray(snap, np.int64)
    flag = np.ascontiguousarray(flag, np.uint8)
    tris = np.ascontiguousarray(tris, np.int32)
    S = np.zeros((H, W), np.uint8)
    frags = np.zeros(1, np.int64); bbox = np.zeros(1, np.int64)
    culled = lib().orc_raster(int(tris.shape[0]), _p(tris), 0, _p(snap), _p(flag), W, H,
                              int(bool(cull_back)), _p(S), _p(frags), _p(bbox))
    return S, int(frags[0]), int(culled), int(bbox[0])


def counts(S, M):
    S = np.ascontiguousarray(S, np.uint8); M = np.ascontiguousarray(M, np.uint8)
    out = np.zeros(4, np.int64)
    lib().orc_counts(S.shape[1], S.shape[0], _p(S), _p(M), _p(out))
    return out


def eval_population(scene, params, mask, cull_back: bool = False, n_threads: int = 1,
                    guard: float = GUARD_PX):
    """Counts for lam candidates.  params [lam, 9*n_instruments]; mask [H,W] 0/1.
    Returns a dict of int64 arrays: s, m, I, xor, frags, culled, flagged, bbox_px."""
    ch = _Chain(scene)
    verts, tris, vframe = _flat_mesh(scene)
    K = scene.K
    params = np.ascontiguousarray(np.asarray(params, np.float64).reshape(-1, 9 * scene.n_instruments))
    lam = params.shape[0]
    mask = np.ascontiguousarray(mask, np.uint8)
    assert mask.shape == (K.height, K.width)
    out = np.zeros((lam, 8), np.int64)
    rc = lib().orc_eval_population(*ch.args(), int(scene.n_instruments), lam, _p(params),
                                   int(verts.shape[0]), _p(verts), _p(vframe), int(tris.shape[0]),
                                   _p(tris), K.fx, K.fy, K.cx, K.cy, K.z_near, guard, K.width,
                                   K.height, int(bool(cull_back)), _p(mask), _p(out), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the chain")
    keys = ["s", "m", "I", "xor", "frags", "culled", "flagged", "bbox_px"]
    return {k: out[:, i].copy() for i, k in enumerate(keys)}


def render(scene, state, guard: float = GUARD_PX):
    """Union silhouette [H,W] of one candidate (all instruments)."""
    K = scene.K
    S = np.zeros((K.height, K.width), np.uint8)
    _, tris, _ = _flat_mesh(scene)
    state = np.asarray(state, np.float64)
    for b in range(scene.n_instruments):
        pr = project(scene, state[9 * b: 9 * b + 9], guard)
        Sb, _, _, _ = raster(pr["snap"], pr["flag"], tris, K.width, K.height)
        S |= Sb
    return S


def loss_from_counts(kind: int, s, m, I, lambda_app: float = 0.0):
    """Losses in FP32, IEEE round-to-nearest, from integer counts.

    kind 0 XOR = s + m - 2I (the MSE term of Eq. render_loss for binary images);
    kind 1 1 - IoU with IoU = I / (s + m - I), 0 when the union is empty (the
    mask error of Sec. IV-B); kind 2 MSE + lambda_app |s - m| (Eq. render_loss,
    appearance term read as |sum S - sum M|)."""
    s = np.asarray(s, np.int64); m = np.asarray(m, np.int64); I = np.asarray(I, np.int64)
    xor = s + m - 2 * I
    if kind == 0:
        return xor.astype(np.float32)
    if kind == 1:
        U = s + m - I
        with np.errstate(invalid="ignore", divide="ignore"):
            q = np.where(U > 0, I.astype(np.float32) / np.maximum(U, 1).astype(np.float32),
                         np.float32(1.0)).astype(np.float32)
        return (np.float32(1.0) - q).astype(np.float32)
    if kind == 2:
        app = np.abs(s - m).astype(np.float32)
        return (xor.astype(np.float32) + np.float32(lambda_app) * app).astype(np.float32)
    raise ValueError(kind)
