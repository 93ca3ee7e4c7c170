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


def test_noalloc_allocates_nothing(api):
    """The defining property: the call takes no device memory.  Free device
    memory is the same before and after a call (outputs made beforehand; the
    first call may load the library's kernels on the device, so the second is
    measured)."""
    from paper_2603_11404_gb300._abi import call
    sc = wl.make_scene("c2", "c2")
    rng = np.random.default_rng(2001)
    gt = wl.sample_state(rng, sc.K)
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    tr = api.Tracker(sc, loss_kind=wl.LOSS_ONE_MINUS_IOU, lambda_max=64)
    Mp = tr.pack_mask(torch.from_numpy(M).cuda())
    v4, t4 = _device_mesh(sc)
    P = torch.from_numpy(wl.population_around(rng, gt, 64)).cuda()
    loss = torch.empty(64, dtype=torch.float32, device="cuda")
    counts = torch.empty((64, 4), dtype=torch.int32, device="cuda")
    ch, Ki, cfg = _structs(sc, wl.LOSS_ONE_MINUS_IOU)
    args = (C.c_void_p(v4.data_ptr()), v4.shape[0], C.c_void_p(t4.data_ptr()), t4.shape[0], C.byref(ch),
            C.byref(Ki), C.byref(cfg), C.c_void_p(P.data_ptr()), 64, C.c_void_p(Mp.data_ptr()),
            C.c_void_p(loss.data_ptr()), C.c_void_p(counts.data_ptr()), None)
    call("eval_population_noalloc", *args)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call("eval_population_noalloc", *args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref_loss, ref_counts = tr.eval_population(P, Mp, counts=True)
    assert torch.equal(counts, ref_counts)


def test_noalloc_rejects_what_tracker_create_rejects(api):
    """The host-side checks of tracker_create, plus the population's limit."""
    from paper_2603_11404_gb300._abi import TrkError, call
    sc = wl.make_scene("c1", "c1")
    v4, t4 = _device_mesh(sc)
    Mp = torch.zeros((sc.K.height, (sc.K.width + 31) // 32), dtype=torch.int32, device="cuda")
    P = torch.zeros((2, 9), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")

    def attempt(n_verts=None, n_tris=None, lam=2, edit=lambda ch, K, cfg: None):
        ch, Ki, cfg = _structs(sc, wl.LOSS_XOR)
        edit(ch, Ki, cfg)
        with pytest.raises(TrkError) as e:
            call("eval_population_noalloc", C.c_void_p(v4.data_ptr()), v4.shape[0] if n_verts is None else n_verts,
                 C.c_void_p(t4.data_ptr()), t4.shape[0] if n_tris is None else n_tris, C.byref(ch), C.byref(Ki),
                 C.byref(cfg), C.c_void_p(P.data_ptr()), lam, C.c_void_p(Mp.data_ptr()), C.c_void_p(out.data_ptr()),
                 None, None)
        assert e.value.status == 1  # TRK_EINVAL: nothing was enqueued

    attempt(n_tris=(1 << 24) + 1)
    attempt(n_verts=(1 << 24) + 1)
    attempt(lam=70000)
    attempt(edit=lambda ch, K, cfg: setattr(K, "fx", float("inf")))
    attempt(edit=lambda ch, K, cfg: setattr(K, "z_near", float("nan")))
    attempt(edit=lambda ch, K, cfg: ch.offset[1].__setitem__(2, float("nan")))
    attempt(edit=lambda ch, K, cfg: ch.coef.__setitem__(1, float("inf")))
    attempt(edit=lambda ch, K, cfg: ch.q_lb.__setitem__(0, 2.0))  # lower limit above the upper one


def test_noalloc_culls_out_of_range_device_indices(api):
    """Indices in the caller's device memory are checked by the kernel: a
    vertex whose frame index is out of range is flagged and a triangle with a
    vertex index out of range is not drawn; both count as culled.  The result
    equals the tracker-based evaluation of the mesh without those triangles."""
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(71)
    gt = wl.sample_state(rng, sc.K)
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    verts, tris, vframe = sc.flat()
    V, nF = verts.shape[0], len(sc.frames)
    # a visible shaft vertex and a visible shaft triangle (frame 0 holds the shaft)
    bad_v = int(np.nonzero(vframe == 0)[0][len(np.nonzero(vframe == 0)[0]) // 2])
    touching = np.nonzero((tris == bad_v).any(axis=1))[0]
    bad_t = int(np.setdiff1d(np.arange(tris.shape[0] // 2, tris.shape[0]), touching)[0])
    v4, t4 = _device_mesh(sc)
    v4[bad_v, 3] = float(nF)        # one frame past the last
    t4[bad_t, 1] = V                # one vertex past the last
    gone = set(touching.tolist()) | {bad_t}
    # the reference: the same scene without the affected triangles
    meshes, base = [], 0
    for m in sc.meshes:
        keep = [k for k in range(len(m.tris)) if base_t(sc, m) + k not in gone]
        meshes.append(wl.LinkMesh(m.frame, m.verts, np.asarray(m.tris)[keep]))
    ref = wl.Scene(sc.frames, meshes, sc.q_lb, sc.q_ub, sc.K)
    tr = api.Tracker(ref, loss_kind=wl.LOSS_XOR, lambda_max=16)
    Mp = tr.pack_mask(torch.from_numpy(M).cuda())
    P = torch.from_numpy(wl.population_around(rng, gt, 16)).cuda()
    ref_loss, ref_counts = tr.eval_population(P, Mp, counts=True)
    loss, counts = _noalloc(sc, v4, t4, P, Mp, wl.LOSS_XOR)
    ref_counts = ref_counts.cpu().numpy()
    assert np.array_equal(counts[:, :3], ref_counts[:, :3])
    assert np.array_equal(counts[:, 3], ref_counts[:, 3] + len(gone))
    assert np.array_equal(loss.view(np.int32), ref_loss.cpu().numpy().view(np.int32))


def base_t(sc, mesh):
    """Index of mesh's first triangle in the scene's flat triangle list."""
    base = 0
    for m in sc.meshes:
        if m is mesh:
            return base
        base += len(m.tris)
    raise ValueError("mesh not in scene")
