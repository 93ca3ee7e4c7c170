"""Shared helpers for the tests (no arithmetic of the method lives here)."""
import numpy as np

import oracle
from paper_2603_11404_gb300 import workload as wl

INT32_MIN = np.iinfo(np.int32).min


def scene_tris(scene):
    _, tris, _ = scene.flat()
    return tris


def oracle_counts_from_snapped(scene, snap_c, mask, cull=False):
    """Oracle raster of one candidate given the kernel's snapped vertices
    [n_inst*V, 2] int32 (INT32_MIN = flagged): returns (s, I, m, culled, S)."""
    K = scene.K
    V = scene.n_verts
    tris = scene_tris(scene)
    S = np.zeros((K.height, K.width), np.uint8)
    culled = 0
    for b in range(scene.n_instruments):
        sn = snap_c[b * V:(b + 1) * V].astype(np.int64)
        flag = (snap_c[b * V:(b + 1) * V, 0] == INT32_MIN).astype(np.uint8)
        Sb, _, cb, _ = oracle.raster(sn, flag, tris, K.width, K.height, cull)
        S |= Sb
        culled += cb
    s, m, I, _ = oracle.counts(S, mask)
    return int(s), int(I), int(m), int(culled), S


def tiny_scene(W, H, fx=100.0, verts=None, tris=None):
    """A single rigid mesh (frame 0) for special cases."""
    K = wl.Intrinsics(fx, fx, W / 2, H / 2, W, H)
    sc = wl.Scene(wl.instrument_frames(), [wl.LinkMesh(0, np.asarray(verts, np.float32),
                                                       np.asarray(tris, np.int32))],
                  wl.Q_LB.copy(), wl.Q_UB.copy(), K)
    return sc


def random_mask(rng, H, W, p=0.3):
    return (rng.random((H, W)) < p).astype(np.uint8)
