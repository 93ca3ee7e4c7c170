"""Parity of the CUDA fitness path (eval_population) with the CPU oracle.

Coverage counts must be bit-exact given the kernel's snapped vertices; the
kernel's projection must agree with the FP64 oracle to 1e-4 px; its snapped
coordinates must equal the oracle's except where 256 (u - cx) lies within
1e-3 of a rounding boundary; losses must equal the FP32 formula applied to the
counts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_11404_gb300 import workload as wl

from _helpers import INT32_MIN, oracle_counts_from_snapped, random_mask, tiny_scene

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


RASTERS = [1, 2]  # TRK_RASTER_CLUSTER, TRK_RASTER_BINNED


def _check_population(api, scene, P, M, loss_kind=wl.LOSS_XOR, cull=False, lambda_max=None, lambda_app=0.0,
                      cluster=0, threads=0, fk_tol=1e-4, raster=0):
    lam = P.shape[0]
    tr = api.Tracker(scene, loss_kind=loss_kind, lambda_max=lambda_max or max(lam, 1), cull_backfaces=cull,
                     lambda_app=lambda_app, cluster=cluster, block_threads=threads, raster=raster)
    Md = torch.from_numpy(M).cuda()
    Mp = tr.pack_mask(Md)
    Pd = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
    loss, counts, snap, uv = tr.eval_population_debug(Pd, Mp)
    loss2, counts2 = tr.eval_population(Pd, Mp, counts=True)
    torch.cuda.synchronize()
    loss, counts, snap, uv = loss.cpu().numpy(), counts.cpu().numpy(), snap.cpu().numpy(), uv.cpu().numpy()
    assert np.array_equal(counts, counts2.cpu().numpy())
    assert np.array_equal(loss.view(np.int32), loss2.cpu().numpy().view(np.int32))
    V = scene.n_verts
    n_snap_diff = 0
    for k in range(lam):
        # 1) raster + reduction: bit-exact given the kernel's snapped vertices
        s, I, m, culled, _ = oracle_counts_from_snapped(scene, snap[k], M, cull)
        assert (counts[k] == [s, I, m, culled]).all(), (k, counts[k], (s, I, m, culled))
        # 2) loss formula on those counts
        want = oracle.loss_from_counts(loss_kind, s, m, I, lambda_app)
        assert loss[k].view(np.int32) == np.float32(want).view(np.int32), (k, loss[k], want)
        # 3) kinematics + projection against the FP64 oracle
        for b in range(scene.n_instruments):
            pr = oracle.project(scene, P[k, 9 * b:9 * b + 9].astype(np.float64))
            ok = pr["flag"] == 0
            g_flag = snap[k, b * V:(b + 1) * V, 0] == INT32_MIN
            assert np.array_equal(g_flag, ~ok)
            err = np.abs(uv[k, b * V:(b + 1) * V][ok] - pr["uv"][ok]).max() if ok.any() else 0.0
            assert err <= fk_tol, (k, b, err)
            diff = (snap[k, b * V:(b + 1) * V][ok] != pr["snap"][ok]).any(axis=1)
            if diff.any():
                frac = np.abs(256 * pr["uv"][ok][diff] - np.round(256 * pr["uv"][ok][diff]))
                assert (np.abs(frac - 0.5) < 1e-3).all()
                n_snap_diff += int(diff.sum())
    return counts, loss, n_snap_diff


def test_pack_mask_roundtrip(api):
    sc = wl.make_scene("c1", "c1", K=wl.Intrinsics(200, 200, 50, 38.5, 100, 77))
    tr = api.Tracker(sc)
    rng = np.random.default_rng(0)
    M = random_mask(rng, 77, 100)
    Mp = tr.pack_mask(torch.from_numpy(M).cuda())
    assert Mp.shape == (77, 4)
    back = api.unpack_mask(Mp, 100).cpu().numpy()
    assert np.array_equal(back, M)
    pad = (Mp[:, 3].cpu().numpy().view(np.uint32) >> (100 - 96))
    assert (pad == 0).all()  # bits past W are zero


@pytest.mark.parametrize("raster", RASTERS)
@pytest.mark.parametrize("rot", [wl.ROT_AXIS_ANGLE, wl.ROT_LOOKAT])
def test_c1_population_parity(api, rot, raster):
    sc = wl.make_scene("c1", "c1", rot_param=rot)
    rng = np.random.default_rng(1000)
    gt = wl.sample_state(rng, sc.K, rot_param=rot)
    M = oracle.render(sc, gt)
    P = wl.population_around(rng, gt, 16)
    counts, loss, _ = _check_population(api, sc, P, M, wl.LOSS_XOR, raster=raster)
    assert counts[:, 0].min() > 100  # the tool is in view


@pytest.mark.parametrize("loss_kind", [wl.LOSS_XOR, wl.LOSS_ONE_MINUS_IOU, wl.LOSS_MSE_APP])
def test_loss_kinds_with_corrupted_mask(api, loss_kind):
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(11)
    gt = wl.sample_state(rng, sc.K)
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    P = wl.population_around(rng, gt, 24)
    _check_population(api, sc, P, M, loss_kind, lambda_app=0.37)


@pytest.mark.parametrize("raster", RASTERS)
def test_c2_population_parity(api, raster):
    """640x512, ~20k triangles, lam = 64, 1 - IoU: the metric's configuration
    (the binned form draws its densest tiles in several work items and merges
    them)."""
    sc = wl.make_scene("c2", "c2")
    rng = np.random.default_rng(2000)
    gt = wl.sample_state(rng, sc.K)
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    P = wl.population_around(rng, gt, 64)
    counts, loss, nd = _check_population(api, sc, P, M, wl.LOSS_ONE_MINUS_IOU, raster=raster)
    assert nd <= 2


@pytest.mark.parametrize("raster", RASTERS)
def test_bimanual_and_ragged_image(api, raster):
    K = wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77)
    sc = wl.make_scene("c1", "c1", n_instruments=2, K=K)
    rng = np.random.default_rng(5)
    gt = np.concatenate([wl.sample_state(rng, K), wl.sample_state(rng, K)])
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    P = wl.population_around(rng, gt, 7)
    _check_population(api, sc, P, M, wl.LOSS_ONE_MINUS_IOU, lambda_max=9, raster=raster)


def test_branched_chain_matches_oracle(api):
    """A chain other than the instrument's: eight frames whose levels (distance
    from a root) hold 2, 2, 3 and 1 frames, so the level-by-level composition
    takes two passes on one level; a small mesh on every frame."""
    F = wl.Frame
    frames = [F(-1, (0.0, 0.0, 0.0)), F(-1, (0.0, 0.0, 0.0), 1, 0, 1.0), F(1, (0.0, 0.0, 9.0), 2, 1, 1.0),
              F(2, (3.0, 0.0, 2.0), 2, 2, 0.5), F(2, (-3.0, 0.0, 2.0), 2, 2, -0.5), F(2, (0.0, 3.0, 2.0), 3, 2, 1.0),
              F(3, (0.0, 0.0, 4.0), 1, 1, 0.7), F(1, (0.0, 4.0, 0.0))]
    meshes = [wl.shaft_mesh(0, length=60.0, rings=6)] + [wl.box_mesh(f, 3.0, 2.0, 4.0, div=(1, 1, 2)) for f in range(1, 8)]
    K = wl.Intrinsics(200.0, 200.0, 80.0, 64.0, 160, 128)
    sc = wl.Scene(frames, meshes, wl.Q_LB.copy(), wl.Q_UB.copy(), K)
    rng = np.random.default_rng(17)
    gt = wl.sample_state(rng, K)
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    assert M.sum() > 200
    P = wl.population_around(rng, gt, 6)
    _check_population(api, sc, P, M, wl.LOSS_ONE_MINUS_IOU)


@pytest.mark.parametrize("raster", RASTERS)
def test_largest_image(api, raster):
    """1280 x 1280, the largest image a tracker takes (a 200 KB bitmap per CTA
    in the cluster form, 20 x 40 tiles in the binned form), with the
    5000-triangle mesh close to the camera."""
    K = wl.Intrinsics(1600.0, 1600.0, 640.0, 640.0, 1280, 1280)
    sc = wl.make_scene("5000", "c1", K=K)
    rng = np.random.default_rng(37)
    gt = wl.sample_state(rng, K, z_range=(60.0, 90.0))
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    P = wl.population_around(rng, gt, 3)
    counts, _, _ = _check_population(api, sc, P, M, wl.LOSS_ONE_MINUS_IOU, raster=raster)
    assert counts[:, 0].min() > 10000


@pytest.mark.parametrize("raster", RASTERS)
def test_single_candidate_and_cull_mode(api, raster):
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(6)
    gt = wl.sample_state(rng, sc.K)
    M = oracle.render(sc, gt)
    P = wl.population_around(rng, gt, 1)
    _check_population(api, sc, P, M, cull=True, raster=raster)


@pytest.mark.parametrize("raster", RASTERS)
@pytest.mark.parametrize("cluster,threads", [(1, 32), (1, 64), (2, 128), (8, 256), (3, 96)])
def test_launch_shapes_agree(api, cluster, threads, raster):
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(7)
    gt = wl.sample_state(rng, sc.K)
    M = oracle.render(sc, gt)
    P = wl.population_around(rng, gt, 5)
    _check_population(api, sc, P, M, cluster=cluster, threads=threads, raster=raster)


@pytest.mark.parametrize("raster", RASTERS)
@pytest.mark.parametrize("cluster,threads", [(1, 64), (4, 64), (2, 96)])
def test_bimanual_launch_shapes_agree(api, cluster, threads, raster):
    """Two instruments with one or two warps beyond the composing ones (with
    64 threads every warp composes and also clears the bitmap)."""
    K = wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77)
    sc = wl.make_scene("c1", "c1", n_instruments=2, K=K)
    rng = np.random.default_rng(27)
    gt = np.concatenate([wl.sample_state(rng, K), wl.sample_state(rng, K)])
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    P = wl.population_around(rng, gt, 4)
    _check_population(api, sc, P, M, wl.LOSS_ONE_MINUS_IOU, cluster=cluster, threads=threads, raster=raster)


@pytest.mark.parametrize("raster", RASTERS)
def test_large_triangles_warp_path(api, raster):
    """Near-camera close-up: triangles wider than 32 px go to the warp path."""
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(8)
    gt = wl.sample_state(rng, sc.K)
    gt[3:6] = [0.0, 0.0, 25.0]
    M = random_mask(rng, sc.K.height, sc.K.width)
    P = wl.population_around(rng, gt, 6, sigma_mm=0.5)
    counts, _, _ = _check_population(api, sc, P, M, raster=raster)
    assert counts[:, 0].max() > 2000


@pytest.mark.parametrize("raster", RASTERS)
def test_full_screen_quad_and_overflow(api, raster):
    """Two triangles covering all W*H pixel centres, plus many large triangles
    (more than the deferred-list capacity, so the CTA redraws every large
    triangle after its loop)."""
    W, H, fx, z = 64, 48, 100.0, 100.0
    # corners at pixel (-0.5, -0.5) .. (W-0.5, H-0.5) on the plane z (vertex frame = E, pose t = (0,0,z))
    x0, x1 = (-0.5 - W / 2) * z / fx, (W - 0.5 - W / 2) * z / fx
    y0, y1 = (-0.5 - H / 2) * z / fx, (H - 0.5 - H / 2) * z / fx
    quad = [[x0, y0, 0], [x1, y0, 0], [x1, y1, 0], [x0, y1, 0]]
    verts = list(quad)
    tris = [[0, 1, 2], [0, 2, 3]]
    rng = np.random.default_rng(9)
    for _ in range(3000):  # ~65 % wider than 32 px: more than one CTA's 1024-entry deferred list
        c = rng.uniform([x0, y0], [x1, y1])
        base = len(verts)
        for _k in range(3):
            verts.append([c[0] + rng.uniform(-40, 40), c[1] + rng.uniform(-15, 15), 0.0])
        tris.append([base, base + 1, base + 2])
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0]], np.float32)
    M = random_mask(rng, H, W)
    counts, _, _ = _check_population(api, sc, st, M, cluster=1, threads=256, raster=raster)
    assert counts[0, 0] == W * H


def test_deferred_list_overflow_draws_every_large_triangle(api):
    """About 2000 thin triangles 40-60 px wide on one CTA: more than its
    1024-entry deferred list, so the CTA redraws every large triangle after the
    loop; the union covers only part of the image, so a triangle left out
    would change the counts (checked bit for bit against the oracle)."""
    W, H, fx, z = 512, 256, 100.0, 100.0
    rng = np.random.default_rng(19)
    verts, tris = [], []
    for _ in range(2000):
        cx_, cy_ = rng.uniform(-W / 2, W / 2), rng.uniform(-H / 2, H / 2)  # px offsets from the centre
        w_, h_ = rng.uniform(40, 60), rng.uniform(0.5, 2.0)
        base = len(verts)
        for dx, dy in ((-w_ / 2, 0.0), (w_ / 2, -h_), (w_ / 2, h_)):
            verts.append([(cx_ + dx) * z / fx, (cy_ + dy) * z / fx, 0.0])
        tris.append([base, base + 1, base + 2])
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0], [0, 0, 0.01, 0.3, -0.2, z, 0, 0, 0]], np.float32)
    M = random_mask(rng, H, W)
    counts, _, _ = _check_population(api, sc, st, M, cluster=1, threads=256)
    assert 0.2 * W * H < counts[0, 0] < 0.9 * W * H  # not saturated: every triangle matters


def test_binned_pool_overflow_draws_tiles_from_every_triangle(api):
    """A fan of 200 sectors (radius 650 px) of a disc in a 1024 x 1024 image:
    each sector's box touches about 70 of the 512 tiles, 14k bin entries in
    all, more than a candidate's pool holds (three per triangle + 8192), so
    every tile is drawn from all triangles instead.  The fan is watertight
    (fragments = union, checked on the oracle) and covers 85 % of the image,
    so a sector left out or drawn twice would change the counts."""
    W, H, fx, z = 1024, 1024, 100.0, 100.0
    n, R = 200, 650.0
    ax, ay = 300.0 - W / 2, 500.0 - H / 2
    verts = [[ax * z / fx, ay * z / fx, 0.0]]
    for t in np.linspace(0, 2 * np.pi, n + 1)[:-1]:
        verts.append([(ax + R * np.cos(t)) * z / fx, (ay + R * np.sin(t)) * z / fx, 0.0])
    tris = [[0, 1 + k, 1 + (k + 1) % n] for k in range(n)]
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0], [0, 0, 0.02, 5.0, -3.0, z, 0, 0, 0]], np.float32)
    rng = np.random.default_rng(41)
    M = random_mask(rng, H, W)
    for raster in RASTERS:
        counts, _, _ = _check_population(api, sc, st, M, raster=raster)
        assert 0.8 * W * H < counts[0, 0] < 0.9 * W * H


def test_rasterisers_agree_on_tracking_workload(api):
    """The two rasterisers give identical counts and losses on 640x512
    populations of several trajectory frames (and so identical CMA-ES runs)."""
    sc = wl.make_scene("c2", "c2")
    rng = np.random.default_rng(2024)
    gt0 = wl.sample_state(rng, sc.K)
    traj = wl.sinusoidal_trajectory(rng, gt0, 4)
    trs = [api.Tracker(sc, loss_kind=wl.LOSS_ONE_MINUS_IOU, lambda_max=64, raster=r) for r in RASTERS]
    for f in range(4):
        M = torch.from_numpy(wl.corrupt_mask(oracle.render(sc, traj[f]), rng)).cuda()
        P = torch.from_numpy(wl.population_around(rng, traj[f], 64)).cuda()
        out = [tr.eval_population(P, tr.pack_mask(M), counts=True) for tr in trs]
        assert torch.equal(out[0][1], out[1][1])
        assert torch.equal(out[0][0].view(torch.int32), out[1][0].view(torch.int32))


@pytest.mark.parametrize("raster", RASTERS)
def test_all_vertices_flagged_and_nan(api, raster):
    from paper_2603_11404_gb300._abi import TRK_DEVERR_NONFINITE
    sc = wl.make_scene("c1", "c1")
    rng = np.random.default_rng(10)
    M = random_mask(rng, sc.K.height, sc.K.width)
    P = np.zeros((3, 9), np.float32)
    P[0, 5] = -50.0          # behind the camera
    P[1, :] = np.nan         # non-finite state
    P[2, 3] = 1e6; P[2, 5] = 100.0  # far outside the guard band
    tr = api.Tracker(sc, lambda_max=3, raster=raster)
    Mp = tr.pack_mask(torch.from_numpy(M).cuda())
    assert tr.get_error() == 0
    loss, counts = tr.eval_population(torch.from_numpy(P[[0, 2]]).cuda(), Mp, counts=True)
    assert tr.get_error() == 0  # flagged vertices alone are no error
    loss, counts = tr.eval_population(torch.from_numpy(P).cuda(), Mp, counts=True)
    counts = counts.cpu().numpy()
    assert (counts[:, 0] == 0).all() and (counts[:, 1] == 0).all()
    assert (counts[:, 3] == sc.n_tris).all()
    assert (loss.cpu().numpy() == M.sum()).all()
    # the NaN state is reported as a warning in the device error word, then cleared
    assert tr.get_error() == TRK_DEVERR_NONFINITE
    assert tr.get_error() == 0


def test_empty_population_and_limits(api):
    sc = wl.make_scene("c1", "c1")
    tr = api.Tracker(sc, lambda_max=4)
    Mp = torch.zeros((sc.K.height, tr.words_per_row), dtype=torch.int32, device="cuda")
    out = tr.eval_population(torch.zeros((0, 9), dtype=torch.float32, device="cuda"), Mp)
    assert out.numel() == 0
    from paper_2603_11404_gb300._abi import TrkError
    with pytest.raises(TrkError):
        tr.eval_population(torch.zeros((5, 9), dtype=torch.float32, device="cuda"), Mp)


def test_render_matches_oracle(api):
    sc = wl.make_scene("c2", "c2")
    rng = np.random.default_rng(12)
    gt = wl.sample_state(rng, sc.K).astype(np.float32)
    tr = api.Tracker(sc, lambda_max=1)
    S = api.unpack_mask(tr.render(torch.from_numpy(gt).cuda()), sc.K.width).cpu().numpy()
    Mz = np.zeros_like(S)
    _, _, snap, _ = tr.eval_population_debug(torch.from_numpy(gt[None]).cuda(),
                                             torch.zeros((sc.K.height, tr.words_per_row), dtype=torch.int32,
                                                         device="cuda"))
    _, _, _, _, S_or = oracle_counts_from_snapped(sc, snap[0].cpu().numpy(), Mz)
    assert np.array_equal(S, S_or)
    assert S.sum() > 1000


def test_repeat_launches_deterministic(api):
    sc = wl.make_scene("c2", "c2")
    rng = np.random.default_rng(13)
    gt = wl.sample_state(rng, sc.K)
    M = torch.from_numpy(wl.corrupt_mask(oracle.render(sc, gt), rng)).cuda()
    tr = api.Tracker(sc, loss_kind=wl.LOSS_ONE_MINUS_IOU, lambda_max=64)
    Mp = tr.pack_mask(M)
    P = torch.from_numpy(wl.population_around(rng, gt, 64)).cuda()
    ref = tr.eval_population(P, Mp, counts=True)[1].clone()
    for _ in range(5):
        assert torch.equal(tr.eval_population(P, Mp, counts=True)[1], ref)


def _lattice_quads(rng, W, H, n, z, fx, corner_px=True):
    """n quadrilaterals, each two triangles (a, b, c), (a, c, d) sharing a-c,
    with corners on pixel centres (or on the 1/256 px lattice near them), so
    that edges and diagonals run through pixel centres: the top-left rule
    decides many pixels on both the outer edges and the shared diagonal."""
    verts, tris = [], []
    for _ in range(n):
        cu, cv = rng.integers(4, W - 4), rng.integers(4, H - 4)
        pts = []
        for ang in np.sort(rng.uniform(0, 2 * np.pi, 4)):
            r = rng.integers(1, 6)
            du, dv = np.round(r * np.cos(ang)), np.round(r * np.sin(ang))
            if not corner_px:
                du += rng.integers(-3, 4) / 256.0
                dv += rng.integers(-3, 4) / 256.0
            pts.append(((cu + du - W / 2) * z / fx, (cv + dv - H / 2) * z / fx, 0.0))
        base = len(verts)
        verts.extend(pts)
        if rng.random() < 0.5:  # either diagonal, either winding
            q = [base, base + 1, base + 2, base + 3]
        else:
            q = [base + 1, base + 2, base + 3, base]
        if rng.random() < 0.5:
            q = q[::-1]
        tris.append([q[0], q[1], q[2]])
        tris.append([q[0], q[2], q[3]])
    return verts, tris


@pytest.mark.parametrize("corner_px", [True, False])
def test_quad_pairs_on_the_pixel_lattice(api, corner_px):
    """Pairs of triangles drawn as one quadrilateral: corners, edges and shared
    diagonals through pixel centres (corner_px) or 1/256 px beside them; convex
    and non-convex pairs of both windings (a non-convex pair is drawn as two
    triangles).  Bit-exact against the oracle's triangle-by-triangle union,
    with and without back-face culling."""
    W, H, fx, z = 96, 64, 100.0, 100.0
    rng = np.random.default_rng(61 + corner_px)
    verts, tris = _lattice_quads(rng, W, H, 400, z, fx, corner_px)
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0], [0, 0, 0, 3.0 / 256, -5.0 / 256, z, 0, 0, 0]], np.float32)
    M = random_mask(rng, H, W)
    for cull in (False, True):
        for cluster, threads in ((1, 32), (2, 128), (8, 256)):
            _check_population(api, sc, st, M, cull=cull, cluster=cluster, threads=threads)


def test_quad_pairs_folded_degenerate_and_flagged(api):
    """Pairs that must not be drawn as one quadrilateral: the second triangle
    folded back over the first (a silhouette edge seen from the side), the
    fourth corner on the diagonal's line (a zero-area second triangle), a
    repeated corner, and pairs with a corner behind the near plane (each
    triangle then counts as culled on its own)."""
    W, H, fx, z = 80, 60, 100.0, 100.0
    rng = np.random.default_rng(67)
    verts, tris = [], []
    for k in range(300):
        cu, cv = rng.uniform(-W / 2 + 6, W / 2 - 6), rng.uniform(-H / 2 + 6, H / 2 - 6)
        a = np.array([cu, cv]); c = a + rng.uniform(-5, 5, 2); b = a + rng.uniform(-5, 5, 2)
        kind = k % 4
        if kind == 0:  # folded: d on b's side of a-c
            d = b + 0.3 * (c - b) + rng.uniform(-0.5, 0.5, 2)
        elif kind == 1:  # d on the line a-c, beyond c
            d = a + 1.5 * (c - a)
        elif kind == 2:  # d repeats b
            d = b.copy()
        else:  # a regular pair, one corner pushed behind the camera below
            d = a + c - b
        base = len(verts)
        for p in (a, b, c, d):
            zz = z
            verts.append([p[0] * zz / fx, p[1] * zz / fx, 0.0])
        if kind == 3 and k % 8 == 3:
            verts[base + 3][2] = -150.0  # z = 100 - 150 < z_near
        tris.append([base, base + 1, base + 2])
        tris.append([base, base + 2, base + 3])
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0], [0.01, -0.02, 0.03, 0.4, -0.3, z, 0, 0, 0]], np.float32)
    M = random_mask(rng, H, W)
    counts, _, _ = _check_population(api, sc, st, M)
    assert (counts[:, 3] > 0).all()  # the flagged pairs were counted per triangle
    _check_population(api, sc, st, M, cull=True)



def test_large_quads_deferred_over_the_cluster(api):
    """Large quadrilaterals (boxes of 100-3000 px, many wider than 32 px, so
    that they go to the deferred list and are drawn after the loop by warps of
    every CTA of the cluster) mixed with records that draw nothing (off-screen
    pairs); bit-exact against the oracle, with and without culling, on one CTA
    and on a cluster of eight."""
    W, H, fx, z = 160, 128, 100.0, 100.0
    rng = np.random.default_rng(73)
    verts, tris = [], []
    for k in range(600):
        if k % 3 == 2:  # a pair far off screen: nothing to draw
            cu, cv, r = rng.uniform(-4 * W, -2 * W), rng.uniform(-H, H), 3.0
        else:
            cu, cv = rng.uniform(-W / 2, W / 2), rng.uniform(-H / 2, H / 2)
            r = rng.choice([6.0, 12.0, 20.0, 28.0])
        ang = np.sort(rng.uniform(0, 2 * np.pi, 4))
        base = len(verts)
        for t_ in ang:
            verts.append([(cu + r * np.cos(t_)) * z / fx, (cv + r * np.sin(t_)) * z / fx, 0.0])
        q = [base, base + 1, base + 2, base + 3]
        if rng.random() < 0.5:
            q = q[::-1]
        tris.append([q[0], q[1], q[2]])
        tris.append([q[0], q[2], q[3]])
    sc = tiny_scene(W, H, fx, verts, tris)
    st = np.array([[0, 0, 0, 0, 0, z, 0, 0, 0], [0.0, 0.0, 0.3, 2.0, -1.0, z, 0, 0, 0]], np.float32)
    M = random_mask(rng, H, W)
    for cull in (False, True):
        for cluster, threads in ((1, 64), (8, 256)):
            _check_population(api, sc, st, M, cull=cull, cluster=cluster, threads=threads)
