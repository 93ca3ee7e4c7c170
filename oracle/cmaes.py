"""FP64 CMA-ES, the optimiser of Sec. III-A.1 (oracle side; test infrastructure).

Mean and covariance updates are Eq. (cmaes_update):
    mu'    = mu + c_m sum_{i<=K} w_i (Theta_i - mu)
    Sigma' = (1 - c_1 - c_mu) Sigma + c_1 p_c p_c^T
             + c_mu sum_{i<=K} w_i y_i y_i^T,      y_i = (Theta_i - mu) / sigma
over the K best of lam samples, ranked only by fitness (Sec. III-A.1).  The
paper leaves the weights, learning rates, the evolution paths and the step-size
rule to the cited CMA-ES; they follow N. Hansen, "The CMA Evolution Strategy:
A Tutorial" (arXiv:1604.00772), with these readings:

* K = floor(lam / 2), w_i proportional to ln((lam + 1)/2) - ln i, sum w = 1,
  mu_eff = 1 / sum w^2; c_sigma, d_sigma, c_c, c_1, c_mu at the tutorial's
  defaults for n = d; c_m = 1.  Both c_m and c_mu accept overrides (the paper
  raises them without giving values, Sec. IV).
* The step size follows cumulative step-size adaptation with path p_sigma and
  the stall indicator h_sigma; Sigma's update carries the tutorial's
  (1 - h_sigma) c_1 c_c (2 - c_c) correction (zero when h_sigma = 1, which
  reduces to the paper's equation).
* The search runs in normalised coordinates x = Theta / scales (Sec. IV:
  "the parameter space is normalized"), Sigma^(0) = I.
* Samples are y_k = C^(1/2) z_k with the symmetric square root
  C^(1/2) = B diag(sqrt(ev)) B^T.  This has the tutorial's distribution
  N(0, C) (the tutorial writes B D z) but does not depend on how an
  eigensolver orders or signs eigenvectors, so two implementations agree
  sample by sample.  C^(-1/2) is formed the same way.
* Ranking ties are broken by candidate index (stable sort on (loss, k)).
* Block-diagonal mode (Sec. III-B): mu, sigma, p_sigma and p_c stay shared over
  the 18-vector; Sigma is updated by the same formula and its off-diagonal
  9x9 blocks are held at zero, so each arm's block evolves from its own
  sub-vectors.  The constants use n = d.

The normals z come from ``philox.normals(seed, stream, generation_total, lam*d)``.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox


def default_constants(n: int, lam: int, c_m: float = 1.0, c_mu_scale: float = 1.0):
    mu = lam // 2
    wp = np.log((lam + 1) / 2.0) - np.log(np.arange(1, mu + 1))
    w = wp / wp.sum()
    mu_eff = 1.0 / np.sum(w * w)
    c_sigma = (mu_eff + 2.0) / (n + mu_eff + 5.0)
    d_sigma = 1.0 + 2.0 * max(0.0, math.sqrt((mu_eff - 1.0) / (n + 1.0)) - 1.0) + c_sigma
    c_c = (4.0 + mu_eff / n) / (n + 4.0 + 2.0 * mu_eff / n)
    c_1 = 2.0 / ((n + 1.3) ** 2 + mu_eff)
    c_mu = min(1.0 - c_1, 2.0 * (mu_eff - 2.0 + 1.0 / mu_eff) / ((n + 2.0) ** 2 + mu_eff))
    c_mu = min(1.0 - c_1, c_mu * c_mu_scale)
    chi_n = math.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n))
    return dict(mu=mu, w=w, mu_eff=mu_eff, c_sigma=c_sigma, d_sigma=d_sigma, c_c=c_c, c_1=c_1,
                c_mu=c_mu, c_m=c_m, chi_n=chi_n)


def _sym_pow(C: np.ndarray, p: float, block: int = 0) -> np.ndarray:
    """C^p for symmetric positive definite C (per diagonal block if block > 0)."""
    if block:
        out = np.zeros_like(C)
        for b0 in range(0, C.shape[0], block):
            sl = slice(b0, b0 + block)
            out[sl, sl] = _sym_pow(C[sl, sl], p)
        return out
    ev, B = np.linalg.eigh(C)
    return (B * ev ** p) @ B.T


class CMAES:
    def __init__(self, d: int, lam: int, mean_phys, scales, sigma0: float = 1.0, seed: int = 0,
                 stream: int = 0, block_diag: bool = False, c_m: float = 1.0,
                 c_mu_scale: float = 1.0):
        self.d, self.lam = d, lam
        self.scales = np.asarray(scales, np.float64).copy()
        self.sigma0 = float(sigma0)
        self.seed, self.stream = int(seed), int(stream)
        self.block = 9 if block_diag else 0
        self.k = default_constants(d, lam, c_m, c_mu_scale)
        self.gen_total = 0
        self.reset(mean_phys)

    def reset(self, mean_phys, sigma0: float | None = None):
        """Start a new search around mean_phys: Sigma = I, sigma = sigma0, paths 0."""
        self.m = np.asarray(mean_phys, np.float64) / self.scales
        self.sigma = self.sigma0 if sigma0 is None else float(sigma0)
        self.C = np.eye(self.d)
        self.p_sigma = np.zeros(self.d)
        self.p_c = np.zeros(self.d)
        self.gen = 0
        self.best_loss = np.inf
        self.best_x = None

    def normals(self):
        """The standard normals of the next generation [lam, d]."""
        return philox.normals(self.seed, self.stream, self.gen_total, self.lam * self.d).reshape(self.lam, self.d)

    def ask(self, z=None):
        """Sample lam candidates (from the given normals z [lam, d], else the
        generator's).  Returns FP32 physical params [lam, d]."""
        self.z = self.normals() if z is None else np.asarray(z, np.float64).reshape(self.lam, self.d)
        self.C_half = _sym_pow(self.C, 0.5, self.block)
        self.y = self.z @ self.C_half.T
        self.x = self.m[None, :] + self.sigma * self.y
        self.params = (self.x * self.scales[None, :]).astype(np.float32)
        return self.params

    def tell(self, loss):
        """Update from the fitness of the last ask (lower is better)."""
        k = self.k
        loss = np.asarray(loss)
        order = np.lexsort((np.arange(self.lam), loss))  # by loss, then index
        if loss[order[0]] < self.best_loss:
            self.best_loss = float(loss[order[0]])
            self.best_x = self.params[order[0]].copy()
        ysel = self.y[order[: k["mu"]]]
        yw = k["w"] @ ysel
        self.m = self.m + k["c_m"] * self.sigma * yw
        C_inv_half = _sym_pow(self.C, -0.5, self.block)
        cs, n = k["c_sigma"], self.d
        self.p_sigma = (1 - cs) * self.p_sigma + math.sqrt(cs * (2 - cs) * k["mu_eff"]) * (C_inv_half @ yw)
        ps_norm = float(np.linalg.norm(self.p_sigma))
        h_sigma = 1.0 if ps_norm / math.sqrt(1 - (1 - cs) ** (2 * (self.gen + 1))) < \
            (1.4 + 2.0 / (n + 1)) * k["chi_n"] else 0.0
        cc = k["c_c"]
        self.p_c = (1 - cc) * self.p_c + h_sigma * math.sqrt(cc * (2 - cc) * k["mu_eff"]) * yw
        c1, cmu = k["c_1"], k["c_mu"]
        delta = (1 - h_sigma) * cc * (2 - cc)
        rank_mu = (ysel.T * k["w"]) @ ysel
        C = (1 + c1 * delta - c1 - cmu) * self.C + c1 * np.outer(self.p_c, self.p_c) + cmu * rank_mu
        if self.block:
            mask = np.zeros_like(C)
            for b0 in range(0, self.d, self.block):
                mask[b0:b0 + self.block, b0:b0 + self.block] = 1
            C = C * mask
        self.C = 0.5 * (C + C.T)
        self.sigma = self.sigma * math.exp((cs / k["d_sigma"]) * (ps_norm / k["chi_n"] - 1))
        self.gen += 1
        self.gen_total += 1
        self.h_sigma = h_sigma
        return order

    @property
    def mean_phys(self):
        return self.m * self.scales

    def state(self):
        return dict(m=self.m.copy(), sigma=self.sigma, C=self.C.copy(), p_sigma=self.p_sigma.copy(),
                    p_c=self.p_c.copy(), gen=self.gen, gen_total=self.gen_total)
