"""The rule the fitness kernel uses for edge-sharing triangle pairs, checked on
the CPU against the oracle's triangle-by-triangle union.

The kernel draws two triangles (a, b, c) and (a, c, d) that share the edge a-c,
have the same orientation and form a strictly convex quadrilateral as one
quadrilateral: a pixel centre is covered when the four edge functions of
(a, b, c, d) in positive orientation pass the top-left rule.  The argument:
under the top-left rule a centre p is covered exactly when p + (e, e^2),
e -> 0+, lies strictly inside, that point never lies on the diagonal, and the
open quadrilateral minus the diagonal is the union of the two open triangles.
These tests state the quadrilateral rule in a few lines of numpy (written here,
not taken from the CUDA sources) and compare it with the oracle's raster of the
two triangles on random convex pairs whose corners, edges and diagonals run
through pixel centres or lie 1/256 px beside them, and check that the pairs
the rule must refuse (non-convex, folded) do differ from their union.
"""
import numpy as np
import pytest

import oracle

SUB = 256


def _orient(p, q, r):
    return (q[0] - p[0]) * (r[1] - p[1]) - (r[0] - p[0]) * (q[1] - p[1])


def _convex_pair(a, b, c, d):
    A1, A2 = _orient(a, b, c), _orient(a, c, d)
    Da, Dc = _orient(b, d, a), _orient(b, d, c)
    return ((A1 > 0 and A2 > 0) or (A1 < 0 and A2 < 0)) and ((Da > 0 > Dc) or (Da < 0 < Dc))


def _quad_raster(a, b, c, d, W, H):
    """Pixels of a convex quadrilateral under the top-left rule on its four
    edges (corners put in positive orientation first)."""
    pts = [a, b, c, d]
    if _orient(a, b, c) < 0:
        pts = [a, d, c, b]
    jj, ii = np.meshgrid(np.arange(W, dtype=np.int64) * SUB, np.arange(H, dtype=np.int64) * SUB)
    cov = np.ones((H, W), bool)
    for k in range(4):
        (x0, y0), (x1, y1) = pts[k], pts[(k + 1) % 4]
        dx, dy = x1 - x0, y1 - y0
        bias = 0 if (dy < 0 or (dy == 0 and dx > 0)) else 1
        cov &= dx * (ii - y0) - dy * (jj - x0) - bias >= 0
    return cov.astype(np.uint8)


def _tri_union(a, b, c, d, W, H):
    pts = np.array([a, b, c, d], np.int64)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    S, _, _, _ = oracle.raster(pts, np.zeros(4, np.uint8), tris, W, H)
    return S


def _random_pair(rng, W, H, lattice):
    cu, cv = rng.integers(3, W - 3), rng.integers(3, H - 3)
    angs = np.sort(rng.uniform(0, 2 * np.pi, 4))
    out = []
    for t in angs:
        r = rng.integers(1, 4)
        x, y = cu + round(r * np.cos(t)), cv + round(r * np.sin(t))
        X, Y = x * SUB, y * SUB
        if not lattice:
            X += int(rng.integers(-2, 3))
            Y += int(rng.integers(-2, 3))
        out.append((X, Y))
    if rng.random() < 0.5:
        out = out[::-1]
    return out


@pytest.mark.parametrize("lattice", [True, False])
def test_convex_pairs_equal_their_union(lattice):
    rng = np.random.default_rng(101 + lattice)
    W, H = 16, 14
    checked = 0
    for _ in range(1500):
        a, b, c, d = _random_pair(rng, W, H, lattice)
        if not _convex_pair(a, b, c, d):
            continue
        assert np.array_equal(_quad_raster(a, b, c, d, W, H), _tri_union(a, b, c, d, W, H)), (a, b, c, d)
        checked += 1
    assert checked > 500


def test_refused_pairs_are_not_their_quadrilateral():
    """A folded pair (d on b's side of a-c) and a dart (a reflex corner) are not
    drawn as one quadrilateral; for each there are centres where the
    quadrilateral rule and the union disagree, so the convexity test matters."""
    W, H = 16, 14
    S = SUB
    folded = ((2 * S, 2 * S), (10 * S, 3 * S), (4 * S, 11 * S), (9 * S, 6 * S))   # d inside triangle abc
    dart = ((2 * S, 2 * S), (12 * S, 7 * S), (2 * S, 12 * S), (5 * S, 7 * S))      # reflex corner at d
    for q in (folded, dart):
        assert not _convex_pair(*q)
        assert not np.array_equal(_quad_raster(*q, W, H), _tri_union(*q, W, H))
