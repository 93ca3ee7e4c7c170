"""The oracle tracker fits the 160x128 single-instrument workload (CPU only)."""
import numpy as np

import oracle
from oracle.cmaes import CMAES
from oracle.tracker import track_frame
from paper_2603_11404_gb300 import workload as wl


def test_c1_fit_reduces_xor():
    sc = wl.make_scene("c1", "c1")
    ratios = []
    for k in range(4):
        rng = np.random.default_rng(1000 + k)
        gt = wl.sample_state(rng, sc.K)
        M = oracle.render(sc, gt)
        init = wl.population_around(rng, gt, 1)[0].astype(np.float64)
        x0 = oracle.eval_population(sc, init[None], M)["xor"][0]
        es = CMAES(9, 16, init, wl.default_scales(9), sigma0=1.0, seed=k)
        best, best_loss = track_frame(es, sc, M, 20, wl.LOSS_XOR, init)
        # the reported best is what it claims to be
        assert oracle.eval_population(sc, best[None], M)["xor"][0] == best_loss
        ratios.append(best_loss / max(x0, 1))
    assert np.median(ratios) < 0.3
