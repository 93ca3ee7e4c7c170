"""The allocation-free entry point (eval_population_noalloc) gives the same
losses and counts as eval_population.

Some callers cannot allocate device memory where they evaluate a population
(code running inside another framework's memory pool, real-time loops that
must not take the allocator's locks, hosts that only hand out pre-registered
buffers).  For them the library offers a call that takes every input and
output from the caller and keeps its one scratch buffer in a fixed device
array.  These tests call it through the C ABI twice in a row and compare with
the tracker-based entry point bit for bit (counts are integers; losses are the
same FP32 formula of the same counts).  This file is collected last so that a
run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2603_11404_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11404_gb300 import build
    build.build()
    from paper_2603_11404_gb300 import api as a
    return a


def _structs(scene, loss_kind, cluster=0, threads=0):
    from paper_2603_11404_gb300 import _abi
    ch = _abi.Chain()
    ch.n_frames = len(scene.frames)
    for f, fr in enumerate(scene.frames):
        ch.parent[f] = fr.parent
        for k in range(3):
            ch.offset[f][k] = float(fr.offset[k])
        ch.axis[f], ch.joint[f], ch.coef[f] = fr.axis, fr.joint, float(fr.coef)
    for i in range(3):
        ch.q_lb[i], ch.q_ub[i] = float(scene.q_lb[i]), float(scene.q_ub[i])
    ch.rot_param, ch.n_instruments = int(scene.rot_param), int(scene.n_instruments)
    K = scene.K
    Ki = _abi.Intrinsics(K.fx, K.fy, K.cx, K.cy, K.width, K.height, K.z_near)
    cfg = _abi.Config(loss_kind, 0.0, 0, 0, cluster, threads)
    return ch, Ki, cfg


def _device_mesh(scene):
    verts, tris, vframe = scene.flat()
    v4 = np.concatenate([verts, vframe[:, None].astype(np.float32)], axis=1).astype(np.float32)
    t4 = np.concatenate([tris, np.zeros((tris.shape[0], 1), np.int32)], axis=1).astype(np.int32)
    return torch.from_numpy(np.ascontiguousarray(v4)).cuda(), torch.from_numpy(np.ascontiguousarray(t4)).cuda()


def _noalloc(scene, v4, t4, P, Mp, loss_kind, cluster=0, threads=0):
    from paper_2603_11404_gb300._abi import call
    ch, Ki, cfg = _structs(scene, loss_kind, cluster, threads)
    lam = P.shape[0]
    loss = torch.full((lam,), -1.0, dtype=torch.float32, device="cuda")
    counts = torch.full((lam, 4), -1, dtype=torch.int32, device="cuda")
    call("eval_population_noalloc", C.c_void_p(v4.data_ptr()), v4.shape[0], C.c_void_p(t4.data_ptr()), t4.shape[0],
         C.byref(ch), C.byref(Ki), C.byref(cfg), C.c_void_p(P.data_ptr()), lam, C.c_void_p(Mp.data_ptr()),
         C.c_void_p(loss.data_ptr()), C.c_void_p(counts.data_ptr()),
         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return loss.cpu().numpy(), counts.cpu().numpy()


@pytest.mark.parametrize("which", ["c2", "bimanual"])
def test_noalloc_matches_eval_population_twice(api, which):
    if which == "c2":
        sc = wl.make_scene("c2", "c2")
        rng = np.random.default_rng(2000)
        gt = wl.sample_state(rng, sc.K)
        lam, kind = 64, wl.LOSS_ONE_MINUS_IOU
    else:
        sc = wl.make_scene("c1", "c1", n_instruments=2, K=wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77))
        rng = np.random.default_rng(5)
        gt = np.concatenate([wl.sample_state(rng, sc.K), wl.sample_state(rng, sc.K)])
        lam, kind = 9, wl.LOSS_XOR
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    tr = api.Tracker(sc, loss_kind=kind, lambda_max=lam)
    Mp = tr.pack_mask(torch.from_numpy(M).cuda())
    v4, t4 = _device_mesh(sc)
    for call_no in range(2):  # two calls in a row: the shared scratch is fully rewritten each time
        P = torch.from_numpy(wl.population_around(rng, gt, lam)).cuda()
        ref_loss, ref_counts = tr.eval_population(P, Mp, counts=True)
        torch.cuda.synchronize()
        loss, counts = _noalloc(sc, v4, t4, P, Mp, kind)
        assert np.array_equal(counts, ref_counts.cpu().numpy()), call_no
        assert np.array_equal(loss.view(np.int32), ref_loss.cpu().numpy().view(np.int32)), call_no
        assert counts[:, 0].max() > 0


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    from paper_2603_11404_gb300._abi import TrkError, TRK_MAX_LAMBDA
    sc = wl.make_scene("c2", "c2")
    v4, t4 = _device_mesh(sc)
    lam = (1 << 21) // sc.n_verts + 1  # one candidate too many for the fixed array
    P = torch.zeros((lam, 9), dtype=torch.float32, device="cuda")
    Mp = torch.zeros((sc.K.height, (sc.K.width + 31) // 32), dtype=torch.int32, device="cuda")
    with pytest.raises(TrkError) as e:
        _noalloc(sc, v4, t4, P, Mp, wl.LOSS_XOR)
    assert "TRK_NOALLOC_MAX_SNAP" in str(e.value)
