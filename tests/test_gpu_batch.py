"""Heterogeneous batches: one persistent launch per generation over instances of
different image sizes, meshes, instrument counts and population sizes gives
exactly the per-instance results."""
import numpy as np
import pytest

import oracle
from oracle import keypoints as okp
from paper_2603_11404_gb300 import workload as wl

from _helpers import random_mask, tiny_scene

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


def _instances(api):
    specs = [
        ("c1", "c1", 1, wl.LOSS_XOR, 16, None),
        ("c2", "c2", 1, wl.LOSS_ONE_MINUS_IOU, 64, None),
        ("c1", "c1", 2, wl.LOSS_ONE_MINUS_IOU, 32, wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77)),
        ("5000", "c2", 1, wl.LOSS_MSE_APP, 48, wl.Intrinsics(400.0, 400.0, 160.0, 128.0, 320, 256)),
    ]
    out = []
    for k, (mesh, cam, ni, loss, lam, K) in enumerate(specs):
        sc = wl.make_scene(mesh, cam, n_instruments=ni, K=K)
        rng = np.random.default_rng(300 + k)
        gt = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(ni)])
        M = wl.corrupt_mask(oracle.render(sc, gt), rng)
        tr = api.Tracker(sc, loss_kind=loss, lambda_max=lam, lambda_app=0.25)
        Mp = tr.pack_mask(torch.from_numpy(M).cuda())
        out.append(dict(sc=sc, gt=gt, tr=tr, Mp=Mp, lam=lam, rng=rng))
    return out


def test_batch_eval_matches_single(api):
    inst = _instances(api)
    P = [torch.from_numpy(wl.population_around(x["rng"], x["gt"], x["lam"])).cuda() for x in inst]
    b = api.Batch([x["tr"] for x in inst], lams=[x["lam"] for x in inst])
    for shape in [(8, 256), (4, 128), (1, 256)]:
        b.set_launch(*shape)
        losses, counts = b.eval(P, [x["Mp"] for x in inst])
        torch.cuda.synchronize()
        for x, p, l, c in zip(inst, P, losses, counts):
            rl, rc = x["tr"].eval_population(p, x["Mp"], counts=True)
            assert torch.equal(c, rc), shape
            assert torch.equal(l.view(torch.int32), rl.view(torch.int32)), shape
    c, t, us = b.autotune([x["Mp"] for x in inst], params=P, reps=3)
    assert c in (1, 2, 4, 8) and t in (128, 256) and us > 0
    assert b.launch()[:2] == (c, t)
    losses, counts = b.eval(P, [x["Mp"] for x in inst])
    for x, p, cc in zip(inst, P, counts):
        assert torch.equal(cc, x["tr"].eval_population(p, x["Mp"], counts=True)[1])


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_track_frame_matches_single(api, use_graph):
    inst = _instances(api)
    scales = lambda x: wl.default_scales(x["sc"].d)
    opt_b = [api.CMAES(x["tr"], x["lam"], x["gt"] + 0.01, scales(x), seed=10 + i, block_diag=x["sc"].d == 18)
             for i, x in enumerate(inst)]
    opt_s = [api.CMAES(x["tr"], x["lam"], x["gt"] + 0.01, scales(x), seed=10 + i, block_diag=x["sc"].d == 18)
             for i, x in enumerate(inst)]
    b = api.Batch([x["tr"] for x in inst], optimisers=opt_b)
    for frame in range(3):
        poses = b.track_frame([x["Mp"] for x in inst], 4, use_graph=use_graph)
        torch.cuda.synchronize()
        for x, o, pb in zip(inst, opt_s, poses):
            ps = o.track_frame(x["Mp"], 4)
            torch.cuda.synchronize()
            assert torch.equal(pb, ps), frame
    for ob, os_ in zip(opt_b, opt_s):
        sa, sb = ob.state(), os_.state()
        assert np.array_equal(sa["C"], sb["C"]) and sa["sigma"] == sb["sigma"]


def test_batch_at_the_batching_workload_sizes(api):
    """Instances at the batching workload's extremes (1280x1024 with a 40k-triangle
    mesh, a bi-manual 640x512 scene, a 320x256 5k-triangle scene with lambda = 256)
    in one persistent launch: counts bit-identical to the per-instance launches,
    and sampled candidates of the largest instance equal to the oracle's."""
    specs = [("40000", 1, 32, (1280, 1024)), ("20000", 2, 64, (640, 512)), ("5000", 1, 256, (320, 256))]
    inst = []
    for k, (mesh, ni, lam, (W, H)) in enumerate(specs):
        K = wl.Intrinsics(1.25 * W, 1.25 * W, W / 2, H / 2, W, H)
        sc = wl.make_scene(mesh, "c2", n_instruments=ni, K=K)
        rng = np.random.default_rng(800 + k)
        gt = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(ni)])
        M = wl.corrupt_mask(oracle.render(sc, gt), rng)
        tr = api.Tracker(sc, loss_kind=wl.LOSS_ONE_MINUS_IOU, lambda_max=lam)
        P = wl.population_around(rng, gt, lam)
        inst.append(dict(sc=sc, tr=tr, M=M, Mp=tr.pack_mask(torch.from_numpy(M).cuda()), P=P,
                         Pd=torch.from_numpy(P).cuda()))
    b = api.Batch([x["tr"] for x in inst], lams=[x["P"].shape[0] for x in inst])
    losses, counts = b.eval([x["Pd"] for x in inst], [x["Mp"] for x in inst])
    torch.cuda.synchronize()
    for x, l, c in zip(inst, losses, counts):
        rl, rc = x["tr"].eval_population(x["Pd"], x["Mp"], counts=True)
        assert torch.equal(c, rc) and torch.equal(l.view(torch.int32), rl.view(torch.int32))
    big = inst[0]
    ref = oracle.eval_population(big["sc"], big["P"][[0, 31]], big["M"], n_threads=4)
    c = counts[0].cpu().numpy()[[0, 31]]
    assert np.array_equal(c[:, 0], ref["s"]) and np.array_equal(c[:, 1], ref["I"]) and np.array_equal(c[:, 2], ref["m"])


def test_batch_with_filter_and_keypoints_matches_single(api):
    """Instances with the Kalman filter and the keypoint term switched on (on
    some instances only): batched frames equal the per-instance frames bit for
    bit, filtered estimate and covariance included."""
    inst = _instances(api)
    frames, pts = (3, 4), (wl.JAW_TIP, wl.JAW_TIP)
    for k, x in enumerate(inst):
        if k % 2 == 0:
            x["tr"].set_keypoints(frames, pts, 3.0, 0.01)
            tips = okp.project_keypoints(x["sc"], x["gt"].astype(np.float32).astype(np.float64), frames, pts)
            obs = wl.noisy_detections(tips, x["rng"], sigma_px=2.0, p_invalid=0.0)
            x["tr"].set_keypoint_obs(torch.from_numpy(obs).cuda())

    def make(i, x):
        d = x["sc"].d
        o = api.CMAES(x["tr"], x["lam"], x["gt"] + 0.01, wl.default_scales(d), seed=20 + i, block_diag=d == 18)
        if i != 1:
            s = wl.default_scales(d)
            o.set_filter(1 / 30, (s * 0.5) ** 2, (s * 2.0) ** 2, s ** 2, p_vel0=(s * 10) ** 2, seed_mean=i == 2)
        return o

    opt_b = [make(i, x) for i, x in enumerate(inst)]
    opt_s = [make(i, x) for i, x in enumerate(inst)]
    b = api.Batch([x["tr"] for x in inst], optimisers=opt_b)
    for frame in range(3):
        poses = b.track_frame([x["Mp"] for x in inst], 3)
        torch.cuda.synchronize()
        for x, o, pb in zip(inst, opt_s, poses):
            ps = o.track_frame(x["Mp"], 3)
            torch.cuda.synchronize()
            assert torch.equal(pb, ps), frame
    for ob, os_ in zip(opt_b, opt_s):
        sa, sb = ob.state(), os_.state()
        assert np.array_equal(sa["C"], sb["C"]) and sa["sigma"] == sb["sigma"]
        assert np.array_equal(sa["best_x"], sb["best_x"]) and sa["best_loss"] == sb["best_loss"]


def test_batch_deferred_list_overflow(api):
    """About 2000 thin triangles 40-60 px wide for one CTA per candidate: its
    1024-entry deferred list overflows and the batched launch draws the rest in
    the lanes; counts equal the plain launch's (which the oracle pins) bit for bit."""
    W, H, fx, z = 512, 256, 100.0, 100.0
    rng = np.random.default_rng(19)
    verts, tris = [], []
    for _ in range(2000):
        cx_, cy_ = rng.uniform(-W / 2, W / 2), rng.uniform(-H / 2, H / 2)
        w_, h_ = rng.uniform(40, 60), rng.uniform(0.5, 2.0)
        base = len(verts)
        for dx, dy in ((-w_ / 2, 0.0), (w_ / 2, -h_), (w_ / 2, h_)):
            verts.append([(cx_ + dx) * z / fx, (cy_ + dy) * z / fx, 0.0])
        tris.append([base, base + 1, base + 2])
    sc = tiny_scene(W, H, fx, verts, tris)
    tr = api.Tracker(sc, loss_kind=wl.LOSS_ONE_MINUS_IOU, lambda_max=2, cluster=1, block_threads=256)
    Mp = tr.pack_mask(torch.from_numpy(random_mask(rng, H, W)).cuda())
    P = torch.tensor([[0, 0, 0, 0, 0, z, 0, 0, 0], [0, 0, 0.01, 0.3, -0.2, z, 0, 0, 0]], dtype=torch.float32).cuda()
    b = api.Batch([tr], lams=[2])
    b.set_launch(1, 256)
    losses, counts = b.eval([P], [Mp])
    rl, rc = tr.eval_population(P, Mp, counts=True)
    torch.cuda.synchronize()
    assert torch.equal(counts[0], rc) and torch.equal(losses[0].view(torch.int32), rl.view(torch.int32))
    assert 0.2 * W * H < rc[0, 0].item() < 0.9 * W * H
