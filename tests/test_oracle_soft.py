"""Pins of the FP64 soft-silhouette oracle (signed distance, aggregation, loss
and analytic gradient) against closed forms, brute force, the binary oracle
renderer and central finite differences."""
import math

import numpy as np
import pytest

import oracle
from oracle import soft
from paper_2603_11404_gb300 import workload as wl


def _equilateral(side=10.0, c=(20.0, 15.0)):
    h = side * math.sqrt(3) / 2
    pts = np.array([[c[0] - side / 2, c[1] + h / 3], [c[0] + side / 2, c[1] + h / 3], [c[0], c[1] - 2 * h / 3]])
    A = soft._doubled_area(*pts)
    return pts if A > 0 else pts[[0, 2, 1]]


def test_signed_distance_closed_forms():
    side = 10.0
    tri = _equilateral(side)
    cen = tri.mean(axis=0)
    inradius = side / (2 * math.sqrt(3))
    assert soft.signed_distance(tri, cen[0], cen[1]) == pytest.approx(inradius, rel=1e-12)
    # beyond a vertex, along the direction from the centroid: distance to that vertex
    v = tri[2]
    p = v + (v - cen) / np.linalg.norm(v - cen) * 3.0
    assert soft.signed_distance(tri, p[0], p[1]) == pytest.approx(-3.0, rel=1e-12)
    # outside the middle of an edge, along its outward normal
    mid = (tri[0] + tri[1]) / 2
    n = (mid - cen) / np.linalg.norm(mid - cen)
    p = mid + 2.5 * n
    assert soft.signed_distance(tri, p[0], p[1]) == pytest.approx(-2.5, rel=1e-12)
    p = mid - 0.75 * n  # inside, nearest edge is that one
    assert soft.signed_distance(tri, p[0], p[1]) == pytest.approx(0.75, rel=1e-12)
    assert soft.signed_distance(tri, mid[0], mid[1]) == pytest.approx(0.0, abs=1e-12)


def test_signed_distance_matches_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(20):
        tri = rng.uniform(0, 30, size=(3, 2))
        if abs(soft._doubled_area(*tri)) < 5:
            continue
        if soft._doubled_area(*tri) < 0:
            tri = tri[[0, 2, 1]]
        t = np.linspace(0, 1, 20001)
        bnd = np.concatenate([tri[k] + t[:, None] * (tri[(k + 1) % 3] - tri[k]) for k in range(3)])
        P = rng.uniform(-10, 40, size=(50, 2))
        d = soft.signed_distance(tri, P[:, 0], P[:, 1])
        for p, dp in zip(P, d):
            dist = np.min(np.hypot(bnd[:, 0] - p[0], bnd[:, 1] - p[1]))
            # inside by barycentric signs (independent of the edge functions above)
            T = np.array([[tri[1, 0] - tri[0, 0], tri[2, 0] - tri[0, 0]], [tri[1, 1] - tri[0, 1], tri[2, 1] - tri[0, 1]]])
            l1, l2 = np.linalg.solve(T, p - tri[0])
            inside = l1 >= 0 and l2 >= 0 and l1 + l2 <= 1
            assert dp == pytest.approx(dist if inside else -dist, abs=2e-3)


def test_signed_distance_gradient_matches_finite_differences():
    rng = np.random.default_rng(6)
    tri = np.array([[3.0, 4.0], [21.0, 6.5], [9.0, 19.0]])
    assert soft._doubled_area(*tri) > 0
    P = rng.uniform(-5, 25, size=(200, 2))
    d, g = soft.signed_distance(tri, P[:, 0], P[:, 1], grad=True)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        dp = soft.signed_distance(tri + e.reshape(3, 2), P[:, 0], P[:, 1])
        dm = soft.signed_distance(tri - e.reshape(3, 2), P[:, 0], P[:, 1])
        fd = (dp - dm) / (2 * h)
        # points within 1e-4 of a tie between two features sit on a kink; skip them
        smooth = np.abs(fd - g[:, k]) < 1e-3
        assert smooth.mean() > 0.97
        assert np.allclose(fd[smooth], g[smooth, k], atol=1e-7)


def test_single_triangle_aggregation_is_the_clipped_sigmoid():
    tri = _equilateral(8.0, c=(16.0, 12.0))
    W, H = 40, 30
    S, acc = soft.soft_from_triangles([tri], W, H)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    d = soft.signed_distance(tri, px, py)
    ref = np.where(d >= -14.0, 1.0 / (1.0 + np.exp(-d)), 0.0)
    assert np.allclose(S, ref, atol=1e-14)
    # the reversed winding gives the same silhouette
    S2, _ = soft.soft_from_triangles([tri[[0, 2, 1]]], W, H)
    assert np.array_equal(S, S2)


def test_two_triangles_combine_as_a_probabilistic_union():
    t1 = _equilateral(8.0, c=(12.0, 12.0))
    t2 = _equilateral(6.0, c=(22.0, 14.0))
    W, H = 40, 30
    S1, _ = soft.soft_from_triangles([t1], W, H)
    S2, _ = soft.soft_from_triangles([t2], W, H)
    S, _ = soft.soft_from_triangles([t1, t2], W, H)
    assert np.allclose(S, 1 - (1 - S1) * (1 - S2), atol=1e-14)


def test_sharp_limit_equals_the_binary_oracle_render():
    """As sigma -> 0 the soft silhouette becomes the union of covered pixels:
    rounded, it equals the binary oracle renderer except at pixel centres
    within ~1.4e-2 px of an edge (counted, must be few)."""
    for seed in (1, 2, 3):
        sc = wl.make_scene("c1", "c1")
        rng = np.random.default_rng(seed)
        x = wl.sample_state(rng, sc.K)
        S, _ = soft.soft_render(sc, x, sigma=1e-3)
        hard = oracle.render(sc, x)
        undecided = ((S > 1e-6) & (S < 1 - 1e-6)).sum()
        assert np.abs(np.round(S) - hard).sum() <= undecided + 1
        assert undecided <= 0.02 * hard.sum()  # centres within ~0.014 px of an edge
        assert hard.sum() > 100


@pytest.mark.parametrize("n_inst", [1, 2])
def test_gradient_matches_central_differences(n_inst):
    sc = wl.make_scene("800", "c1", n_instruments=n_inst, K=wl.Intrinsics(120.0, 120.0, 40.0, 32.0, 80, 64))
    rng = np.random.default_rng(40 + n_inst)
    gt = np.concatenate([wl.sample_state(rng, sc.K) for _ in range(n_inst)])
    M = oracle.render(sc, gt)
    s9 = wl.default_scales(9 * n_inst)
    x = gt + rng.normal(size=9 * n_inst) * s9
    # a cutoff further out (sigmoid(-25) ~ 1e-11) makes the cutoff jumps negligible: a tight pin
    L, g = soft.soft_grad(sc, x, M, cutoff=25.0)
    fd = np.array([(soft.soft_loss(sc, x + e, M, cutoff=25.0) - soft.soft_loss(sc, x - e, M, cutoff=25.0))
                   / (2 * e[k]) for k, e in enumerate(np.eye(9 * n_inst) * 1e-5 * s9)])
    assert np.linalg.norm((g - fd) * s9) / np.linalg.norm(fd * s9) < 1e-7
    assert L == pytest.approx(soft.soft_loss(sc, x, M, cutoff=25.0), rel=1e-15)
    # the defined loss (cutoff 14): FP64 central differences, h = 1e-4 in normalised units
    L, g = soft.soft_grad(sc, x, M)
    fd = np.array([(soft.soft_loss(sc, x + e, M) - soft.soft_loss(sc, x - e, M)) / (2 * e[k])
                   for k, e in enumerate(np.eye(9 * n_inst) * 1e-4 * s9)])
    assert np.linalg.norm((g - fd) * s9) / np.linalg.norm(fd * s9) < 1e-3
