"""Oracle tracker: per-frame CMA-ES over the oracle renderer (test infrastructure).

Sec. III-A: every frame starts from the previous frame's estimate (or, for the
joints, from joint readings when available, Sec. III-A) and runs a few CMA-ES
generations (3 in Table I, 5 in the 640x512 tracking workload) over the render
loss.  Readings where the paper is silent:
* each frame restarts the search with Sigma = I, sigma = sigma0 and zero paths
  ("CMA-ES is initialized with covariance Sigma^(0) = I", Sec. IV), around the
  previous estimate;
* the frame's estimate is the best candidate seen over its generations (ties
  to the earlier generation, then the lower index).
"""
from __future__ import annotations

import numpy as np

from . import eval_population, loss_from_counts, qhat_from_q
from .cmaes import CMAES


def track_frame(cma: CMAES, scene, mask, generations: int, loss_kind: int, prev_estimate,
                joint_reading=None, n_threads: int = 1, lambda_app: float = 0.0):
    mean = np.asarray(prev_estimate, np.float64).copy()
    if joint_reading is not None:
        for b in range(scene.n_instruments):
            for i in range(3):
                mean[9 * b + 6 + i] = qhat_from_q(joint_reading[3 * b + i], scene.q_lb[i], scene.q_ub[i])
    cma.reset(mean)
    for _ in range(generations):
        P = cma.ask()
        c = eval_population(scene, P, mask, n_threads=n_threads)
        loss = loss_from_counts(loss_kind, c["s"], c["m"], c["I"], lambda_app)
        cma.tell(loss)
    return cma.best_x.astype(np.float64), cma.best_loss
