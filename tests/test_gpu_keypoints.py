"""Keypoint term on the GPU (Eq. kpts_loss) against the FP64 oracle: the
projected jaw tips and the fitness losses with the term switched on."""
import numpy as np
import pytest

import oracle
from oracle import keypoints as okp
from paper_2603_11404_gb300 import workload as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FRAMES, PTS, TAU, LAM = (3, 4), (wl.JAW_TIP, wl.JAW_TIP), 3.0, 0.01


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_11404_gb300 import build
    build.build()
    from paper_2603_11404_gb300 import api as a
    return a


@pytest.mark.parametrize("n_inst,loss_kind", [(1, wl.LOSS_ONE_MINUS_IOU), (2, wl.LOSS_XOR), (1, wl.LOSS_MSE_APP)])
def test_losses_with_keypoint_term_match_oracle(api, n_inst, loss_kind):
    K = wl.Intrinsics(150.0, 150.0, 50.0, 38.5, 101, 77) if n_inst == 2 else None
    sc = wl.make_scene("c1", "c1", n_instruments=n_inst, K=K)
    rng = np.random.default_rng(120 + n_inst + loss_kind)
    gt = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(n_inst)])
    M = wl.corrupt_mask(oracle.render(sc, gt), rng)
    tr = api.Tracker(sc, loss_kind=loss_kind, lambda_max=32, lambda_app=0.25)
    tr.set_keypoints(FRAMES, PTS, TAU, LAM)
    tips = tr.project_keypoints(torch.from_numpy(gt.astype(np.float32))[None].cuda())[0].cpu().numpy()
    ref_tips = okp.project_keypoints(sc, gt.astype(np.float32).astype(np.float64), FRAMES, PTS)
    assert np.allclose(tips, ref_tips, atol=2e-3)
    obs = wl.noisy_detections(ref_tips, rng, sigma_px=2.0, p_invalid=0.0)
    if n_inst == 2:
        obs[1, 4] = 0.0  # one arm without a valid detection
    tr.set_keypoint_obs(torch.from_numpy(obs).cuda())
    P = wl.population_around(rng, gt, 32)
    loss, counts = tr.eval_population(torch.from_numpy(P).cuda(), tr.pack_mask(torch.from_numpy(M).cuda()),
                                      counts=True)
    loss, counts = loss.cpu().numpy(), counts.cpu().numpy()
    ref = oracle.eval_population(sc, P, M)
    assert np.array_equal(counts[:, 0], ref["s"]) and np.array_equal(counts[:, 1], ref["I"])
    base = oracle.loss_from_counts(loss_kind, ref["s"], ref["m"], ref["I"], 0.25)
    for c in range(P.shape[0]):
        term = okp.keypoint_term(sc, P[c].astype(np.float64), obs, FRAMES, PTS, TAU, LAM)
        assert loss[c] == pytest.approx(float(base[c]) + term, rel=1e-5, abs=1e-4), c
    tr.set_keypoint_obs(None)  # the term switched off again
    off = tr.eval_population(torch.from_numpy(P).cuda(), tr.pack_mask(torch.from_numpy(M).cuda())).cpu().numpy()
    assert np.array_equal(off.view(np.int32), np.asarray(base, np.float32).view(np.int32))
