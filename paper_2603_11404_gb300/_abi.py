"""ctypes declarations of the C ABI in include/tracker.h (argument marshalling only).

The library is built in-tree by ``paper_2603_11404_gb300.build.build()``.  There
is no fallback: if the shared library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB

TRK_MAX_FRAMES = 16
TRK_MAX_INSTRUMENTS = 2
TRK_MAX_D = 18
TRK_MAX_LAMBDA = 1024
TRK_MAX_PIXELS = 1280 * 1280

STATUS = {0: "TRK_OK", 1: "TRK_EINVAL", 2: "TRK_ENOMEM", 3: "TRK_ECUDA", 4: "TRK_EDEVICE", 6: "TRK_EBUSY"}
TRK_DEVERR_WORKLIST, TRK_DEVERR_NONFINITE = 0x1, 0x8


class TrkError(RuntimeError):
    def __init__(self, status: int, fn: str, detail: str):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class LinkMesh(C.Structure):
    _fields_ = [("frame", C.c_int32), ("n_verts", C.c_int32), ("verts", C.c_void_p),
                ("n_tris", C.c_int32), ("tris", C.c_void_p)]


class Chain(C.Structure):
    _fields_ = [("n_frames", C.c_int32), ("parent", C.c_int32 * TRK_MAX_FRAMES),
                ("offset", (C.c_double * 3) * TRK_MAX_FRAMES), ("axis", C.c_int32 * TRK_MAX_FRAMES),
                ("joint", C.c_int32 * TRK_MAX_FRAMES), ("coef", C.c_double * TRK_MAX_FRAMES),
                ("q_lb", C.c_double * 3), ("q_ub", C.c_double * 3), ("rot_param", C.c_int32),
                ("n_instruments", C.c_int32)]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("z_near", C.c_double)]


class Config(C.Structure):
    _fields_ = [("loss_kind", C.c_int32), ("lambda_app", C.c_float), ("cull_backfaces", C.c_int32),
                ("lambda_max", C.c_int32), ("cluster", C.c_int32), ("block_threads", C.c_int32),
                ("raster", C.c_int32)]


class Keypoints(C.Structure):
    _fields_ = [("frame", C.c_int32 * 2), ("point", (C.c_double * 3) * 2), ("tau", C.c_double),
                ("lambda_kpts", C.c_double)]


class Filter(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("seed_mean", C.c_int32), ("dt", C.c_double),
                ("q_pos", C.c_double * TRK_MAX_D), ("q_vel", C.c_double * TRK_MAX_D), ("r", C.c_double * TRK_MAX_D),
                ("p_vel0", C.c_double * TRK_MAX_D)]


class FrameResult(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("stream", C.c_int32), ("d", C.c_int32), ("pose", C.c_float * TRK_MAX_D), ("best_loss", C.c_float),
                ("pad", C.c_int32)]


P = C.c_void_p
I32 = C.c_int32
# name -> argtypes (every function returns trk_status = int)
SIGNATURES = {
    "tracker_create": [P, I32, P, P, P, P],
    "tracker_destroy": [P],
    "tracker_info": [P, P, P, P, P, P, P],
    "tracker_get_error": [P, P, P],
    "tracker_pack_mask": [P, P, P, P],
    "eval_population": [P, P, I32, P, P, P, P],
    "eval_population_debug": [P, P, I32, P, P, P, P, P, P],
    "tracker_render": [P, P, P, P],
    "cmaes_create": [P, I32, P, P, C.c_double, C.c_uint64, C.c_uint32, I32, P],
    "cmaes_destroy": [P],
    "cmaes_reset_device": [P, P, P],
    "cmaes_reset_host": [P, P, P],
    "cmaes_ask": [P, P, P],
    "cmaes_tell": [P, P, P],
    "cmaes_ask_normals": [P, P, P, P],
    "cmaes_last_normals": [P, P, P],
    "cmaes_step": [P, P, P],
    "cmaes_get_state_host": [P, P, P, P, P, P, P, P, P, P, P],
    "cmaes_buffers": [P, P, P, P],
    "track_frame_device": [P, P, I32, P, P, P],
    "track_frame_host": [P, P, I32, P, P, P, P],
    "cmaes_save": [P, P, P, P],
    "cmaes_load": [P, P, C.c_size_t, P],
    "trk_probe_int_issue": [I32, P, P, P],
    "eval_population_noalloc": [P, I32, P, I32, P, P, P, P, I32, P, P, P, P],
    "batch_create": [P, P, P, I32, I32, I32, P],
    "batch_destroy": [P],
    "batch_set_launch": [P, I32, I32],
    "batch_get_launch": [P, P, P, P],
    "batch_eval": [P, P, P, P, P, P],
    "batch_track_frame": [P, P, I32, P, I32, P],
    "batch_autotune": [P, P, P, I32, P, P, P, P],
    "soft_eval": [P, P, I32, P, C.c_float, P, P, P],
    "cmaes_set_filter": [P, P, P],
    "tracker_set_keypoints": [P, P],
    "tracker_set_keypoint_obs": [P, P],
    "tracker_project_keypoints": [P, P, I32, P, P],
    "soft_refine": [P, P, I32, I32, C.c_float, C.c_float, P, P, P],
    "server_create": [I32, I32, I32, C.c_int64, I32, C.c_int64, I32, I32, P],
    "server_destroy": [P],
    "server_add_stream": [P, P, I32, I32, P],
    "server_remove_stream": [P, I32],
    "server_submit": [P, I32, P, P, C.c_uint64, C.c_double],
    "server_step": [P, P, P],
    "server_poll": [P, P, I32, I32, P],
    "server_stats": [P, P, P, P, P],
}

_lib = None
_lock = threading.Lock()


def lib():
    """Load the built library (no fallback: raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"CUDA library not built ({LIB}); run paper_2603_11404_gb300.build.build()")
            L = C.CDLL(LIB)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.trk_status_string.restype = C.c_char_p
            L.trk_status_string.argtypes = [C.c_int]
            L.tracker_last_error.restype = C.c_char_p
            L.tracker_last_error.argtypes = []
            L.server_now.restype = C.c_double
            L.server_now.argtypes = []
            _lib = L
    return _lib


def call(name: str, *args) -> None:
    """Call a status-returning entry point; raise TrkError on failure."""
    L = lib()
    rc = getattr(L, name)(*args)
    if rc != 0:
        raise TrkError(rc, name, L.tracker_last_error().decode(errors="replace"))


def declared_symbols():
    """Every function name declared in include/tracker.h."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tracker.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:trk_status|const char \*|double)\s*(\w+)\s*\(", src, re.M)))
