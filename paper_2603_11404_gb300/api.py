"""Python face of the C ABI: the same entry points, taking torch CUDA tensors.

Every function here only marshals arguments (pointers, sizes, the current
torch stream) into the calls declared in include/tracker.h; all of the work
runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import call

LOSS_XOR, LOSS_ONE_MINUS_IOU, LOSS_MSE_APP = 0, 1, 2
RASTER_AUTO, RASTER_CLUSTER, RASTER_BINNED = 0, 1, 2


# the current stream's handle in one call each (torch.cuda.current_stream()
# builds a Stream object per call, a noticeable share of a frame's host time)
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(stream.cuda_stream)
    if _raw_stream is not None and _cur_device is not None:
        return C.c_void_p(_raw_stream(_cur_device()))
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    raise TypeError(type(t))


def _check_dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


class Tracker:
    """tracker_create(mesh, links, intrinsics) and the fitness entry points."""

    def __init__(self, scene, loss_kind: int = LOSS_XOR, lambda_max: int = 64, cull_backfaces: bool = False,
                 lambda_app: float = 0.0, cluster: int = 0, block_threads: int = 0, raster: int = 0):
        self.scene = scene
        K = scene.K
        self._keep = []
        meshes = (_abi.LinkMesh * len(scene.meshes))()
        for i, m in enumerate(scene.meshes):
            v = np.ascontiguousarray(m.verts, np.float32)
            t = np.ascontiguousarray(m.tris, np.int32)
            self._keep += [v, t]
            meshes[i] = _abi.LinkMesh(int(m.frame), int(v.shape[0]), v.ctypes.data, int(t.shape[0]), t.ctypes.data)
        ch = _abi.Chain()
        ch.n_frames = len(scene.frames)
        for f, fr in enumerate(scene.frames):
            ch.parent[f] = fr.parent
            for k in range(3):
                ch.offset[f][k] = float(fr.offset[k])
            ch.axis[f] = fr.axis
            ch.joint[f] = fr.joint
            ch.coef[f] = float(fr.coef)
        for i in range(3):
            ch.q_lb[i] = float(scene.q_lb[i])
            ch.q_ub[i] = float(scene.q_ub[i])
        ch.rot_param = int(scene.rot_param)
        ch.n_instruments = int(scene.n_instruments)
        Ki = _abi.Intrinsics(float(K.fx), float(K.fy), float(K.cx), float(K.cy), int(K.width), int(K.height),
                             float(K.z_near))
        cfg = _abi.Config(int(loss_kind), float(lambda_app), int(bool(cull_backfaces)), int(lambda_max),
                          int(cluster), int(block_threads), int(raster))
        h = C.c_void_p()
        call("tracker_create", meshes, len(scene.meshes), C.byref(ch), C.byref(Ki), C.byref(cfg), C.byref(h))
        self.h = h
        d, nv, nt, w, hh, wq = (C.c_int32() for _ in range(6))
        call("tracker_info", h, C.byref(d), C.byref(nv), C.byref(nt), C.byref(w), C.byref(hh), C.byref(wq))
        self.d, self.n_verts, self.n_tris = d.value, nv.value, nt.value
        self.width, self.height, self.words_per_row = w.value, hh.value, wq.value
        self.n_instruments = int(scene.n_instruments)
        self.lambda_max = int(lambda_max)
        self.loss_kind = int(loss_kind)

    def get_error(self, stream=None) -> int:
        """tracker_get_error: the device error word's bits (TRK_DEVERR_*), cleared
        by the read; raises TrkError (TRK_EDEVICE) when an error bit was set."""
        w = C.c_uint32()
        call("tracker_get_error", self.h, C.byref(w), _stream(stream))
        return w.value

    def close(self):
        if getattr(self, "h", None):
            call("tracker_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- masks -------------------------------------------------------------
    def pack_mask(self, mask: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """tracker_pack_mask: uint8 [H, W] (nonzero = tool) -> int32 [H, ceil(W/32)] packed rows."""
        _check_dev(mask, torch.uint8, "mask")
        if tuple(mask.shape) != (self.height, self.width):
            raise ValueError("mask shape")
        if out is None:
            out = torch.empty((self.height, self.words_per_row), dtype=torch.int32, device=mask.device)
        call("tracker_pack_mask", self.h, _ptr(mask), _ptr(out), _stream(stream))
        return out

    # -- fitness -----------------------------------------------------------
    def eval_population(self, params: torch.Tensor, mask_packed: torch.Tensor, loss: torch.Tensor | None = None,
                        counts: torch.Tensor | bool | None = None, stream=None):
        """eval_population: params [lam, d] FP32 -> loss [lam] FP32 (and counts [lam, 4] int32:
        s, I, m, culled when counts is True or a tensor)."""
        _check_dev(params, torch.float32, "params")
        _check_dev(mask_packed, torch.int32, "mask_packed")
        lam = params.shape[0] if params.dim() == 2 else 0
        if params.dim() != 2 or params.shape[1] != self.d:
            raise ValueError("params must be [lam, d]")
        if loss is None:
            loss = torch.empty(lam, dtype=torch.float32, device=params.device)
        if counts is True:
            counts = torch.empty((lam, 4), dtype=torch.int32, device=params.device)
        elif counts is False:
            counts = None
        call("eval_population", self.h, _ptr(params), lam, _ptr(mask_packed), _ptr(loss), _ptr(counts),
             _stream(stream))
        return (loss, counts) if counts is not None else loss

    def eval_population_debug(self, params: torch.Tensor, mask_packed: torch.Tensor, stream=None):
        """eval_population_debug: returns loss, counts [lam,4], snapped [lam, n_inst*V, 2] int32,
        uv [lam, n_inst*V, 2] FP32 offsets from the principal point."""
        _check_dev(params, torch.float32, "params")
        lam = params.shape[0]
        dev = params.device
        loss = torch.empty(lam, dtype=torch.float32, device=dev)
        counts = torch.empty((lam, 4), dtype=torch.int32, device=dev)
        nv = self.n_instruments * self.n_verts
        snap = torch.empty((lam, nv, 2), dtype=torch.int32, device=dev)
        uv = torch.empty((lam, nv, 2), dtype=torch.float32, device=dev)
        call("eval_population_debug", self.h, _ptr(params), lam, _ptr(mask_packed), _ptr(loss), _ptr(counts),
             _ptr(snap), _ptr(uv), _stream(stream))
        return loss, counts, snap, uv

    def set_keypoints(self, frames, points, tau: float, lambda_kpts: float):
        """tracker_set_keypoints: two keypoints (frame index, point in mm in that frame)."""
        kp = _abi.Keypoints()
        for k in range(2):
            kp.frame[k] = int(frames[k])
            for j in range(3):
                kp.point[k][j] = float(points[k][j])
        kp.tau, kp.lambda_kpts = float(tau), float(lambda_kpts)
        call("tracker_set_keypoints", self.h, C.byref(kp))

    def set_keypoint_obs(self, obs: torch.Tensor | None):
        """tracker_set_keypoint_obs: device tensor [n_inst, 5] (x1, y1, x2, y2, valid) or None."""
        if obs is not None:
            _check_dev(obs, torch.float32, "obs")
        self._kp_obs = obs
        call("tracker_set_keypoint_obs", self.h, _ptr(obs))

    def project_keypoints(self, states: torch.Tensor, stream=None) -> torch.Tensor:
        """tracker_project_keypoints: [n, d] states -> [n, n_inst, 4] (u1, v1, u2, v2)."""
        _check_dev(states, torch.float32, "states")
        n = states.shape[0]
        out = torch.empty((n, self.scene.n_instruments, 4), dtype=torch.float32, device=states.device)
        call("tracker_project_keypoints", self.h, _ptr(states), n, _ptr(out), _stream(stream))
        return out

    def soft_eval(self, params: torch.Tensor, mask_packed: torch.Tensor, sigma: float = 1.0, grad: bool = False,
                  stream=None):
        """soft_eval: soft-silhouette loss [lam] (and dL/dparams [lam, d] when grad)."""
        _check_dev(params, torch.float32, "params")
        lam = params.shape[0]
        loss = torch.empty(lam, dtype=torch.float32, device=params.device)
        g = torch.empty((lam, self.d), dtype=torch.float32, device=params.device) if grad else None
        call("soft_eval", self.h, _ptr(params), lam, _ptr(mask_packed), float(sigma), _ptr(loss), _ptr(g),
             _stream(stream))
        return (loss, g) if grad else loss

    def render(self, state: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """tracker_render: one state [d] -> packed silhouette int32 [H, ceil(W/32)]."""
        _check_dev(state, torch.float32, "state")
        if out is None:
            out = torch.empty((self.height, self.words_per_row), dtype=torch.int32, device=state.device)
        call("tracker_render", self.h, _ptr(state.reshape(-1).contiguous()), _ptr(out), _stream(stream))
        return out


def unpack_mask(packed: torch.Tensor, width: int) -> torch.Tensor:
    """Packed rows -> uint8 [H, W] (inverse of pack_mask, for inspection and tests)."""
    H, Wq = packed.shape
    bits = torch.arange(32, device=packed.device, dtype=torch.int32)
    u = ((packed.unsqueeze(-1) >> bits) & 1).to(torch.uint8).reshape(H, Wq * 32)
    return u[:, :width].contiguous()


def probe_int_issue(iters: int = 2000) -> dict:
    """trk_probe_int_issue: the measured 32-bit integer issue rate of the current
    device (the fitness kernel's roofline denominator) and the derived figure."""
    tops, ms, derived = C.c_double(), C.c_double(), C.c_double()
    call("trk_probe_int_issue", int(iters), C.byref(tops), C.byref(ms), C.byref(derived))
    return {"tops": tops.value, "ms": ms.value, "derived_tops": derived.value}


class CMAES:
    """Device-resident CMA-ES: cmaes_create / ask / tell / step / track_frame."""

    def __init__(self, tracker: Tracker, lam: int, mean, scales, sigma0: float = 1.0, seed: int = 0,
                 stream_id: int = 0, block_diag: bool = False):
        self.tracker = tracker
        self.lam, self.d = int(lam), tracker.d
        mean = np.ascontiguousarray(mean, np.float64)
        scales = np.ascontiguousarray(scales, np.float64)
        if mean.shape != (self.d,) or scales.shape != (self.d,):
            raise ValueError("mean/scales must have d entries")
        h = C.c_void_p()
        call("cmaes_create", tracker.h, self.lam, _ptr(mean), _ptr(scales), float(sigma0), int(seed) & (2 ** 64 - 1),
             int(stream_id), int(bool(block_diag)), C.byref(h))
        self.h = h
        K = tracker.scene.K
        self._hw = (K.height, K.width)
        self._tfh = _abi.lib().track_frame_host

    def close(self):
        if getattr(self, "h", None):
            call("cmaes_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, mean, stream=None):
        mean = np.ascontiguousarray(mean, np.float64)
        call("cmaes_reset_host", self.h, _ptr(mean), _stream(stream))

    def ask(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.lam, self.d), dtype=torch.float32, device="cuda")
        call("cmaes_ask", self.h, _ptr(out), _stream(stream))
        return out

    def ask_normals(self, z: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """cmaes_ask_normals: sample with caller-supplied standard normals z [lam, d] FP64."""
        _check_dev(z, torch.float64, "z")
        if out is None:
            out = torch.empty((self.lam, self.d), dtype=torch.float32, device="cuda")
        call("cmaes_ask_normals", self.h, _ptr(z), _ptr(out), _stream(stream))
        return out

    def last_normals(self, stream=None) -> torch.Tensor:
        """cmaes_last_normals: the standard normals [lam, d] FP64 of the last population."""
        out = torch.empty((self.lam, self.d), dtype=torch.float64, device="cuda")
        call("cmaes_last_normals", self.h, _ptr(out), _stream(stream))
        return out

    def tell(self, loss: torch.Tensor, stream=None):
        _check_dev(loss, torch.float32, "loss")
        call("cmaes_tell", self.h, _ptr(loss), _stream(stream))

    def step(self, mask_packed: torch.Tensor, stream=None):
        call("cmaes_step", self.h, _ptr(mask_packed), _stream(stream))

    def state(self, stream=None) -> dict:
        d = self.d
        m = np.zeros(d); ps = np.zeros(d); pc = np.zeros(d); Cm = np.zeros(d * d)
        sig = C.c_double(); g = C.c_int32(); gt = C.c_int32()
        bx = np.zeros(d, np.float32); bl = C.c_float()
        call("cmaes_get_state_host", self.h, _ptr(m), C.byref(sig), _ptr(Cm), _ptr(ps), _ptr(pc), C.byref(g),
             C.byref(gt), _ptr(bx), C.byref(bl), _stream(stream))
        return dict(m=m, sigma=sig.value, C=Cm.reshape(d, d), p_sigma=ps, p_c=pc, gen=g.value, gen_total=gt.value,
                    best_x=bx, best_loss=bl.value)

    def track_frame(self, mask_packed: torch.Tensor, generations: int, joint_reading: torch.Tensor | None = None,
                    pose_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """track_frame_device: asynchronous; returns pose_out [d] FP32 on the device."""
        if pose_out is None:
            pose_out = torch.empty(self.d, dtype=torch.float32, device="cuda")
        call("track_frame_device", self.h, _ptr(mask_packed), int(generations), _ptr(joint_reading), _ptr(pose_out),
             _stream(stream))
        return pose_out

    def track_frame_host(self, mask_u8, generations: int, joint_reading=None, stream=None):
        """track_frame_host: host mask [H, W] uint8 (numpy or pinned tensor) -> (pose [d], best loss).
        Kept lean: it runs once per camera frame, so its host time is part of every frame's latency."""
        if isinstance(mask_u8, torch.Tensor):
            if mask_u8.is_cuda or mask_u8.dtype != torch.uint8 or not mask_u8.is_contiguous():
                raise ValueError("mask must be a contiguous host uint8 tensor")
            mp = mask_u8.data_ptr()
        else:
            mask_u8 = np.ascontiguousarray(mask_u8, np.uint8)
            mp = mask_u8.ctypes.data
        if tuple(mask_u8.shape) != self._hw:
            raise ValueError(f"mask must be [{self._hw[0]}, {self._hw[1]}] uint8")
        pose = np.empty(self.d, np.float32)
        bl = C.c_float()
        jp = None
        if joint_reading is not None:
            jr = np.ascontiguousarray(joint_reading, np.float32)
            if jr.size < 3 * self.tracker.scene.n_instruments:
                raise ValueError("joint reading needs 3 values per instrument")
            jp = jr.ctypes.data
        rc = self._tfh(self.h, mp, int(generations), jp, pose.ctypes.data, C.byref(bl), _stream(stream))
        if rc:
            raise _abi.TrkError(rc, "track_frame_host", _abi.lib().tracker_last_error().decode(errors="replace"))
        return pose, bl.value

    def set_filter(self, dt: float, q_pos, q_vel, r, p_vel0=None, seed_mean: bool = True, enabled: bool = True,
                   stream=None):
        """cmaes_set_filter: constant-velocity Kalman filter on the frame estimates
        (per-coordinate arrays, or scalars broadcast to all d coordinates)."""
        f = _abi.Filter()
        f.enabled, f.seed_mean, f.dt = int(bool(enabled)), int(bool(seed_mean)), float(dt)
        arrs = [np.broadcast_to(np.asarray(x, np.float64), (self.d,)) for x in
                (q_pos, q_vel, r, np.full(self.d, 1e2) if p_vel0 is None else p_vel0)]
        for name, a in zip(("q_pos", "q_vel", "r", "p_vel0"), arrs):
            dst = getattr(f, name)
            for i in range(self.d):
                dst[i] = float(a[i])
        call("cmaes_set_filter", self.h, C.byref(f), _stream(stream))

    def refine(self, mask_packed: torch.Tensor, top_k: int = 8, steps: int = 10, lr: float = 0.05,
               sigma: float = 1.0, pose_out: torch.Tensor | None = None, stream=None):
        """soft_refine: Adam steps on the soft loss for the last generation's top_k
        candidates; returns (estimate [d] on the device, index of the adopted
        refined candidate or -1)."""
        if pose_out is None:
            pose_out = torch.empty(self.d, dtype=torch.float32, device="cuda")
        picked = C.c_int32()
        call("soft_refine", self.h, _ptr(mask_packed), int(top_k), int(steps), float(lr), float(sigma),
             _ptr(pose_out), C.byref(picked), _stream(stream))
        return pose_out, picked.value

    def save(self, stream=None) -> bytes:
        n = C.c_size_t()
        call("cmaes_save", self.h, None, C.byref(n), _stream(stream))
        buf = (C.c_char * n.value)()
        call("cmaes_save", self.h, buf, C.byref(n), _stream(stream))
        return bytes(buf)

    def load(self, blob: bytes, stream=None):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        call("cmaes_load", self.h, buf, len(blob), _stream(stream))


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Batch:
    """Heterogeneous batch: batch_create / batch_eval / batch_track_frame / batch_autotune."""

    def __init__(self, trackers, optimisers=None, lams=None, cluster: int = 0, threads: int = 0):
        self.trackers = list(trackers)
        self.optimisers = list(optimisers) if optimisers is not None else None
        n = len(self.trackers)
        th = (C.c_void_p * n)(*[t.h for t in self.trackers])
        oh = None
        lam = None
        if self.optimisers is not None:
            oh = (C.c_void_p * n)(*[o.h for o in self.optimisers])
            self.lams = [o.lam for o in self.optimisers]
        else:
            self.lams = [int(l) for l in lams]
            lam = (C.c_int32 * n)(*self.lams)
        h = C.c_void_p()
        call("batch_create", th, oh, lam, n, int(cluster), int(threads), C.byref(h))
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            call("batch_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch(self):
        c, t, nc = C.c_int32(), C.c_int32(), C.c_int32()
        call("batch_get_launch", self.h, C.byref(c), C.byref(t), C.byref(nc))
        return c.value, t.value, nc.value

    def set_launch(self, cluster: int, threads: int):
        call("batch_set_launch", self.h, int(cluster), int(threads))

    def eval(self, params, masks, stream=None):
        """Per-instance params [lam_i, d_i] and packed masks -> (losses, counts)."""
        losses = [torch.empty(p.shape[0], dtype=torch.float32, device="cuda") for p in params]
        counts = [torch.empty((p.shape[0], 4), dtype=torch.int32, device="cuda") for p in params]
        call("batch_eval", self.h, _ptr_array(params), _ptr_array(masks), _ptr_array(losses), _ptr_array(counts),
             _stream(stream))
        return losses, counts

    def track_frame(self, masks, generations: int, poses=None, use_graph: bool = True, stream=None):
        if poses is None:
            poses = [torch.empty(t.d, dtype=torch.float32, device="cuda") for t in self.trackers]
        self._keep = (list(masks), poses)
        call("batch_track_frame", self.h, _ptr_array(masks), int(generations), _ptr_array(poses), int(bool(use_graph)),
             _stream(stream))
        return poses

    def autotune(self, masks, params=None, reps: int = 5, stream=None):
        c, t, us = C.c_int32(), C.c_int32(), C.c_float()
        call("batch_autotune", self.h, None if params is None else _ptr_array(params), _ptr_array(masks), int(reps),
             C.byref(c), C.byref(t), C.byref(us), _stream(stream))
        return c.value, t.value, us.value


class Server:
    """server_*: camera streams tracked with continuous batching (one CMA-ES
    generation of every admitted frame per tick)."""

    def __init__(self, max_active: int = 8, max_streams: int = 8, max_pending: int = 64,
                 max_pixels: int = 640 * 512, max_lambda: int = 256, hbm_reserve_bytes: int = 0,
                 cluster: int = 0, threads: int = 0):
        h = C.c_void_p()
        call("server_create", int(max_active), int(max_streams), int(max_pending), int(max_pixels), int(max_lambda),
             int(hbm_reserve_bytes), int(cluster), int(threads), C.byref(h))
        self.h = h
        self._out = (_abi.FrameResult * 256)()
        self.optimisers = {}

    def close(self):
        if getattr(self, "h", None):
            call("server_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def now() -> float:
        return _abi.lib().server_now()

    def add_stream(self, cmaes: "CMAES", generations: int, use_joint_reading: bool = False) -> int:
        sid = C.c_int32()
        call("server_add_stream", self.h, cmaes.h, int(generations), int(bool(use_joint_reading)), C.byref(sid))
        self.optimisers[sid.value] = cmaes
        return sid.value

    def remove_stream(self, sid: int):
        call("server_remove_stream", self.h, int(sid))
        self.optimisers.pop(sid, None)

    def submit(self, sid: int, mask_u8: np.ndarray, joint_reading=None, tag: int = 0, t_submit: float = -1.0):
        """Queue a frame; returns False (nothing queued) when the staging pool is full."""
        m = np.ascontiguousarray(mask_u8, np.uint8)
        K = self.optimisers[sid].tracker.scene.K
        if m.shape != (K.height, K.width):
            raise ValueError(f"mask must be [{K.height}, {K.width}] uint8")
        j = None if joint_reading is None else np.ascontiguousarray(joint_reading, np.float32)
        if j is not None and j.size != 3 * self.optimisers[sid].tracker.scene.n_instruments:
            raise ValueError("joint readings must have 3 entries per instrument")
        L = _abi.lib()
        rc = L.server_submit(self.h, int(sid), m.ctypes.data, None if j is None else j.ctypes.data, int(tag),
                             float(t_submit))
        if rc == 6:  # TRK_EBUSY
            return False
        if rc != 0:
            raise _abi.TrkError(rc, "server_submit", L.tracker_last_error().decode(errors="replace"))
        return True

    def step(self):
        """Enqueue one tick; returns (frames in slots, frames waiting)."""
        a, q = C.c_int32(), C.c_int32()
        call("server_step", self.h, C.byref(a), C.byref(q))
        return a.value, q.value

    def poll(self, wait: bool = False):
        out, res = [], self._out
        first = True
        while True:
            n = C.c_int32()
            call("server_poll", self.h, res, len(res), int(bool(wait and first)), C.byref(n))
            first = False
            for i in range(n.value):
                r = res[i]
                out.append(dict(stream=r.stream, tag=r.tag, t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done,
                                pose=np.array(r.pose[:r.d], np.float32), best_loss=r.best_loss))
            if n.value < len(res):
                return out

    def stats(self):
        t, a, q, f = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        call("server_stats", self.h, C.byref(t), C.byref(a), C.byref(q), C.byref(f))
        return dict(ticks=t.value, active=a.value, queued=q.value, free_staging=f.value)

    def run_until_idle(self):
        """Step until every queued frame has finished; returns the results."""
        out = []
        while True:
            a, q = self.step()
            out += self.poll()
            if a == 0 and q == 0:
                break
        return out + self.poll(wait=True)


class SoftSilhouetteLoss(torch.autograd.Function):
    """Soft-silhouette loss per candidate as a differentiable torch op:
    forward = soft_eval without gradient; backward = soft_eval with gradient
    (it recomputes the forward tile by tile), scaled by the incoming grad."""

    @staticmethod
    def forward(ctx, params, tracker, mask_packed, sigma=1.0):
        p = params.detach().contiguous()
        ctx.tracker, ctx.mask, ctx.sigma = tracker, mask_packed, sigma
        ctx.save_for_backward(p)
        return tracker.soft_eval(p, mask_packed, sigma)

    @staticmethod
    def backward(ctx, grad_loss):
        (p,) = ctx.saved_tensors
        _, g = ctx.tracker.soft_eval(p, ctx.mask, ctx.sigma, grad=True)
        return grad_loss.to(g.dtype)[:, None] * g, None, None, None


def soft_silhouette_loss(params: torch.Tensor, tracker: Tracker, mask_packed: torch.Tensor, sigma: float = 1.0):
    return SoftSilhouetteLoss.apply(params, tracker, mask_packed, sigma)
