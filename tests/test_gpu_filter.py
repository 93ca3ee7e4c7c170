"""The device Kalman filter on the frame estimates (temporal filtering,
Sec. III-A) against the FP64 matrix-form oracle fed with the same raw frame
estimates."""
import numpy as np
import pytest

import oracle
from oracle.kalman import Kalman
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


@pytest.mark.parametrize("n_inst,seed_mean", [(1, True), (1, False), (2, True)])
def test_filtered_estimates_match_the_oracle_filter(api, n_inst, seed_mean):
    K = wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77) if n_inst == 2 else None
    sc = wl.make_scene("c1", "c1", n_instruments=n_inst, K=K)
    d = sc.d
    rng = np.random.default_rng(90 + n_inst)
    p0 = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(n_inst)])
    traj = wl.sinusoidal_trajectory(rng, p0, 8)
    tr = api.Tracker(sc, loss_kind=wl.LOSS_XOR, lambda_max=16)
    es = api.CMAES(tr, 16, p0, wl.default_scales(d), sigma0=1.0, seed=5, block_diag=d == 18)
    s = wl.default_scales(d)
    q_pos, q_vel, r = (s * 0.5) ** 2, (s * 2.0) ** 2, s ** 2
    es.set_filter(1 / 30, q_pos, q_vel, r, p_vel0=(s * 10) ** 2, seed_mean=seed_mean)
    kf = Kalman(d, 1 / 30, q_pos, q_vel, r, (s * 10) ** 2, sc.q_lb, sc.q_ub)
    for f in range(8):
        M = oracle.render(sc, traj[f])
        pose = es.track_frame(tr.pack_mask(torch.from_numpy(M).cuda()), 3).cpu().numpy()
        raw = es.state()["best_x"].astype(np.float64)
        if f:
            kf.predict()
        ref = kf.update(raw)
        assert np.allclose(pose, ref.astype(np.float32), rtol=2e-6, atol=2e-6), f
    # joint angles of the estimate are within their limits
    for b in range(n_inst):
        for j in range(3):
            q = oracle.q_from_qhat(float(pose[9 * b + 6 + j]), sc.q_lb[j], sc.q_ub[j])
            assert sc.q_lb[j] - 1e-6 <= q <= sc.q_ub[j] + 1e-6
