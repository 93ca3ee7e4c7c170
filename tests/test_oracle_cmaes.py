"""Pins for the oracle's Philox generator, normals and FP64 CMA-ES (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox
from oracle.cmaes import CMAES, default_constants

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_distribution():
    z = philox.normals(seed=123, stream=4, generation=9, count=200_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct (generation, stream) give unrelated draws
    z2 = philox.normals(seed=123, stream=4, generation=10, count=1000)
    assert abs(np.corrcoef(z[:1000], z2)[0, 1]) < 0.15


def test_weights_and_constants():
    k = default_constants(10, 10)
    assert k["mu"] == 5
    assert abs(k["w"].sum() - 1) < 1e-15 and np.all(np.diff(k["w"]) < 0) and np.all(k["w"] > 0)
    # mu_eff for lam = 10 from the weight definition: about 3.17 (Hansen's tutorial, Table 1 discussion)
    assert abs(k["mu_eff"] - 3.1672) < 1e-3
    for n, lam in [(9, 16), (9, 64), (18, 64), (18, 256)]:
        k = default_constants(n, lam)
        assert 0 < k["c_1"] + k["c_mu"] <= 1 and 0 < k["c_sigma"] < 1 and 0 < k["c_c"] <= 1


# The learning rates at the two benchmark shapes, evaluated by hand from the
# tutorial's default-parameter table (Hansen, arXiv:1604.00772, Table 1) to 30
# digits and written here as literals.  lam = 64: mu = 32 and
#   w'_i = ln(65/2) - ln i (i = 1..32),  mu_eff = (sum w')^2 / sum w'^2 = 17.621652406855657
# (n-independent).  Then, for n = 9 and n = 18:
#   c_sigma = (mu_eff + 2) / (n + mu_eff + 5)            = 0.6205131899622561 | 0.4830343239199235
#   d_sigma = 1 + 2 max(0, sqrt((mu_eff-1)/(n+1)) - 1) + c_sigma
#           (n = 9: sqrt(16.62/10) = 1.289, the max is 0.289; n = 18: sqrt(16.62/19) < 1, 0)
#                                                        = 2.1990129403485661 | 1.4830343239199235
#   c_c     = (4 + mu_eff/n) / (n + 4 + 2 mu_eff/n)      = 0.3522102497214471 | 0.2078215508657473
#   c_1     = 2 / ((n + 1.3)^2 + mu_eff)                 = 0.0161666258682126 | 0.0051267374036655
#   c_mu    = min(1 - c_1, 2 (mu_eff - 2 + 1/mu_eff) / ((n + 2)^2 + mu_eff))
#                                                        = 0.2262042112722312 | 0.0750842332221743
PINNED = {
    (9, 64): dict(mu_eff=17.621652406855657, c_sigma=0.6205131899622561, d_sigma=2.1990129403485661,
                  c_c=0.3522102497214471, c_1=0.0161666258682126, c_mu=0.2262042112722312),
    (18, 64): dict(mu_eff=17.621652406855657, c_sigma=0.4830343239199235, d_sigma=1.4830343239199235,
                   c_c=0.2078215508657473, c_1=0.0051267374036655, c_mu=0.0750842332221743),
}


def _pins_hold(k, n, lam):
    """The constants k match the hand-evaluated values, and chi_n (the
    tutorial's approximation of E|N(0, I)|) is within 2e-4 of the exact
    sqrt(2) Gamma((n+1)/2) / Gamma(n/2)."""
    from scipy.special import gammaln
    want = PINNED[(n, lam)]
    if any(abs(k[key] - v) > 1e-13 * abs(v) for key, v in want.items()):
        return False
    exact = math.sqrt(2.0) * math.exp(gammaln((n + 1) / 2.0) - gammaln(n / 2.0))
    return abs(k["chi_n"] - exact) < 2e-4 * exact


@pytest.mark.parametrize("n,lam", [(9, 64), (18, 64)])
def test_learning_rates_pinned(n, lam):
    assert _pins_hold(default_constants(n, lam), n, lam)


def _planted(n, lam, which):
    """default_constants with one plausible mistake planted (transposed or
    dropped terms); the pins must reject every one of them."""
    k = dict(default_constants(n, lam))
    me = k["mu_eff"]
    if which == "c_sigma":
        k["c_sigma"] = (me + 2.0) / (n + me + 3.0)
    elif which == "d_sigma":
        k["d_sigma"] = 1.0 + 2.0 * max(0.0, math.sqrt((me - 1.0) / (n + 1.0)) - 1.0)
    elif which == "c_c":
        k["c_c"] = (4.0 + me / n) / (n + 4.0 + me / n)
    elif which == "c_1":
        k["c_1"] = 2.0 / ((n + 1.3) + me)
    elif which == "c_mu":
        k["c_mu"] = min(1.0 - k["c_1"], 2.0 * (me - 2.0 + 1.0 / me) / ((n + 1.0) ** 2 + me))
    elif which == "chi_n":
        k["chi_n"] = math.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n))
    elif which == "mu_eff":
        k["mu_eff"] = 1.0 / np.sum(k["w"] ** 3)
    return k


@pytest.mark.parametrize("which", ["c_sigma", "d_sigma", "c_c", "c_1", "c_mu", "chi_n", "mu_eff"])
def test_learning_rate_pins_catch_planted_mistakes(which):
    assert not all(_pins_hold(_planted(n, lam, which), n, lam) for n, lam in PINNED)


def _run(f, d=9, lam=16, gens=200, seed=7, block=False, x0=None, sigma0=0.5):
    es = CMAES(d, lam, np.ones(d) if x0 is None else x0, np.ones(d), sigma0=sigma0, seed=seed,
               block_diag=block)
    hist = []
    for _ in range(gens):
        P = es.ask().astype(np.float64)
        es.tell(np.array([f(p) for p in P]))
        hist.append((es.m.copy(), es.sigma, es.C.copy()))
    return es, hist


def test_rank_only_invariance_bit_identical():
    """Sec. III-A.1: the update uses only the fitness ranking, so a strictly
    monotone transform of the losses leaves the trajectory bit-identical."""
    f = lambda x: float(np.sum((x - 0.3) ** 2 * np.arange(1, 10)))
    _, h1 = _run(f, gens=40)
    _, h2 = _run(lambda x: math.exp(f(x)) + 5.0, gens=40)
    _, h3 = _run(lambda x: f(x) ** 3, gens=40)
    for a, b, c in zip(h1, h2, h3):
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
        assert np.array_equal(a[0], c[0]) and a[1] == c[1] and np.array_equal(a[2], c[2])


def test_sphere_converges_log_linearly():
    es, hist = _run(lambda x: float(np.sum(x * x)), gens=220, sigma0=1.0)
    fvals = [float(np.sum(m * m)) for m, _, _ in hist]
    assert fvals[-1] < 1e-12
    sig = np.log([s for _, s, _ in hist[20:]])
    slope = np.polyfit(np.arange(len(sig)), sig, 1)[0]
    assert -0.2 < slope < -0.02       # steady geometric decrease of sigma
    ev = np.linalg.eigvalsh(hist[-1][2])
    assert ev.max() / ev.min() < 10   # isotropic problem keeps C near-isotropic


def test_ellipsoid_learns_inverse_hessian():
    d = 6
    a = 10.0 ** (3 * np.arange(d) / (d - 1))   # Hessian diag, condition 1e3
    rot = np.linalg.qr(np.random.default_rng(0).normal(size=(d, d)))[0]
    H = rot @ np.diag(a) @ rot.T
    es, hist = _run(lambda x: float(x @ H @ x), d=d, lam=12, gens=400, sigma0=1.0)
    C = hist[-1][2]
    assert float(hist[-1][0] @ H @ hist[-1][0]) < 1e-10
    # C is proportional to H^-1: C H has all eigenvalues equal
    ev = np.linalg.eigvals(C @ H).real
    assert ev.max() / ev.min() < 4.0
    evC = np.linalg.eigvalsh(C)
    assert evC.max() / evC.min() > 100   # it did adapt (condition of H^-1 is 1e3)


def test_covariance_spd_and_block_diagonal():
    f = lambda x: float(np.sum((x - 1) ** 2 * (1 + np.arange(18))))
    es, hist = _run(f, d=18, lam=32, gens=60, block=True)
    for _, _, C in hist:
        assert np.array_equal(C, C.T)
        assert np.all(np.linalg.eigvalsh(C) > 0)
        assert np.all(C[:9, 9:] == 0) and np.all(C[9:, :9] == 0)
    es2, hist2 = _run(f, d=18, lam=32, gens=60, block=False)
    assert np.abs(hist2[-1][2][:9, 9:]).max() > 0   # the full form does couple the arms


def test_linear_function_sigma_grows():
    es, hist = _run(lambda x: float(x[0]), gens=40, sigma0=0.1)
    assert hist[-1][1] > 10 * 0.1


def test_samples_have_covariance_sigma2_C():
    d = 5
    es = CMAES(d, 40000, np.zeros(d), np.ones(d), sigma0=0.7, seed=3)
    A = np.random.default_rng(1).normal(size=(d, d))
    es.C = A @ A.T + np.eye(d)
    P = es.ask().astype(np.float64)
    emp = np.cov(P.T)
    assert np.allclose(emp, 0.49 * es.C, rtol=0.05, atol=0.05 * np.abs(0.49 * es.C).max())
