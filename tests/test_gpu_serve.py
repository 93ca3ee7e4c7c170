"""Serving with continuous batching: every frame's pose is the same whether its
camera stream is served alone, in a mix with other streams (uneven images,
meshes, populations, one or two instruments, with and without joint
readings, fewer slots than streams), or tracked by the plain per-frame call."""
import numpy as np
import pytest

from paper_2603_11404_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_FRAMES = 4


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11404_gb300 import build
    build.build()
    from paper_2603_11404_gb300 import api as a
    return a


SPECS = [  # mesh, camera, instruments, loss, lambda, generations, joint readings, intrinsics
    ("c1", "c1", 1, wl.LOSS_XOR, 16, 3, False, None),
    ("c1", "c1", 2, wl.LOSS_ONE_MINUS_IOU, 32, 2, True, wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77)),
    ("c2", "c2", 1, wl.LOSS_ONE_MINUS_IOU, 64, 2, False, None),
    ("5000", "c2", 1, wl.LOSS_ONE_MINUS_IOU, 48, 4, False, wl.Intrinsics(400.0, 400.0, 160.0, 128.0, 320, 256)),
]


def _streams(api):
    """Per stream: tracker, trajectory, observed masks and joint readings."""
    out = []
    for k, (mesh, cam, ni, loss, lam, gens, joint, K) in enumerate(SPECS):
        sc = wl.make_scene(mesh, cam, n_instruments=ni, K=K)
        rng = np.random.default_rng(700 + k)
        p0 = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(ni)])
        traj = wl.sinusoidal_trajectory(rng, p0, N_FRAMES)
        tr = api.Tracker(sc, loss_kind=loss, lambda_max=lam)
        masks, joints = [], []
        for f in range(N_FRAMES):
            S = api.unpack_mask(tr.render(torch.from_numpy(traj[f].astype(np.float32)).cuda()), sc.K.width)
            masks.append(wl.corrupt_mask(S.cpu().numpy(), rng))
            q = np.concatenate([traj[f][b * 9 + 6: b * 9 + 9] for b in range(ni)])
            joints.append((q + rng.normal(size=q.shape) * 0.02).astype(np.float32) if joint else None)
        out.append(dict(sc=sc, tr=tr, p0=p0, masks=masks, joints=joints, lam=lam, gens=gens, joint=joint, k=k))
    return out


def _optimiser(api, s):
    d = s["sc"].d
    return api.CMAES(s["tr"], s["lam"], s["p0"], wl.default_scales(d), sigma0=0.5, seed=40 + s["k"],
                     block_diag=d == 18)


def _serve(api, streams, max_active):
    srv = api.Server(max_active=max_active, max_streams=len(streams), max_pending=64, max_pixels=640 * 512)
    sids, opts = [], []
    for s in streams:
        o = _optimiser(api, s)
        opts.append(o)
        sids.append(srv.add_stream(o, s["gens"], use_joint_reading=s["joint"]))
    # interleaved submission, frames of every stream in order
    for f in range(N_FRAMES):
        for s, sid in zip(streams, sids):
            assert srv.submit(sid, s["masks"][f], s["joints"][f], tag=f)
    res = srv.run_until_idle()
    assert srv.stats()["free_staging"] == 64
    poses = {}
    for r in res:
        poses[(sids.index(r["stream"]), r["tag"])] = r["pose"]
        assert r["t_submit"] <= r["t_admit"] and r["t_submit"] <= r["t_done"]
    assert len(poses) == len(streams) * N_FRAMES
    return poses, srv


def test_serve_alone_equals_mix_equals_plain(api):
    streams = _streams(api)
    # plain form: per-frame track_frame_host on each stream's own optimiser
    plain = {}
    for j, s in enumerate(streams):
        o = _optimiser(api, s)
        for f in range(N_FRAMES):
            plain[(j, f)] = o.track_frame_host(s["masks"][f], s["gens"], s["joints"][f])[0]
    mix, srv = _serve(api, streams, max_active=3)  # fewer slots than streams: admission waits
    assert srv.stats()["ticks"] >= max(s["gens"] for s in streams) * N_FRAMES
    for j, s in enumerate(streams):
        alone, _ = _serve(api, [s], max_active=1)
        for f in range(N_FRAMES):
            assert np.array_equal(alone[(0, f)], plain[(j, f)]), (j, f)
            assert np.array_equal(mix[(j, f)], plain[(j, f)]), (j, f)


def test_serve_admission_and_back_pressure(api):
    from paper_2603_11404_gb300._abi import TrkError
    s = _streams(api)[0]
    free, total = torch.cuda.mem_get_info()
    srv = api.Server(max_active=2, max_streams=2, max_pending=2, max_pixels=160 * 128, hbm_reserve_bytes=total)
    with pytest.raises(TrkError) as e:  # the reserve can never stay free
        srv.add_stream(_optimiser(api, s), 2)
    assert "TRK_EBUSY" in str(e.value)
    srv = api.Server(max_active=2, max_streams=2, max_pending=2, max_pixels=160 * 128)
    sid = srv.add_stream(_optimiser(api, s), 2)
    assert srv.submit(sid, s["masks"][0], tag=0) and srv.submit(sid, s["masks"][1], tag=1)
    assert not srv.submit(sid, s["masks"][2], tag=2)  # staging pool full
    with pytest.raises(TrkError):
        srv.remove_stream(sid)  # frames still queued
    res = srv.run_until_idle()
    assert sorted(r["tag"] for r in res) == [0, 1]
    srv.remove_stream(sid)
    big = api.Tracker(wl.make_scene("c1", "c2"), lambda_max=16)
    with pytest.raises(TrkError):  # 640x512 image on a 160x128 server
        srv.add_stream(api.CMAES(big, 16, s["p0"], wl.default_scales(9)), 2)
