"""Pins for the oracle's exact integer rasteriser (CPU only).

The oracle's raster is the plain definition of coverage (pixel centres, 1/256
px fixed point, top-left rule).  These tests pin it to things other than
itself: closed-form counts of axis-aligned quads, the full screen, watertight
tessellations, a third implementation in exact rational arithmetic that states
the top-left rule geometrically, and invariances.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

SUB = 256


def _raster(tris_xy, W, H, cull=False):
    """tris_xy: list of ((x,y),(x,y),(x,y)) in 1/256 px."""
    pts = np.array([p for t in tris_xy for p in t], np.int64).reshape(-1, 2)
    tris = np.arange(len(pts), dtype=np.int32).reshape(-1, 3)
    flag = np.zeros(len(pts), np.uint8)
    return oracle.raster(pts, flag, tris, W, H, cull)


def _cdiv(a, b):
    return -((-a) // b)


def _quad_count(X0, Y0, X1, Y1, W, H):
    """Top-left rule on an axis-aligned rectangle: left/top inclusive,
    right/bottom exclusive, so columns ceil(X0/256) .. ceil(X1/256)-1."""
    j0, j1 = max(0, _cdiv(X0, SUB)), min(W, _cdiv(X1, SUB))
    i0, i1 = max(0, _cdiv(Y0, SUB)), min(H, _cdiv(Y1, SUB))
    return max(0, j1 - j0) * max(0, i1 - i0)


def _quad_tris(X0, Y0, X1, Y1, diag, rng):
    a, b, c, d = (X0, Y0), (X1, Y0), (X1, Y1), (X0, Y1)
    tris = [(a, b, c), (a, c, d)] if diag == 0 else [(a, b, d), (b, c, d)]
    out = []
    for t in tris:
        t = list(t)
        r = rng.integers(3)
        t = t[r:] + t[:r]
        if rng.integers(2):
            t = t[::-1]
        out.append(tuple(t))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_axis_aligned_quads_closed_form(seed):
    rng = np.random.default_rng(seed)
    W, H = 37, 29
    for trial in range(60):
        if trial % 3 == 0:   # integer corners: pixel centres on the edges
            X0, X1 = sorted(rng.integers(-3, W + 3, 2) * SUB)
            Y0, Y1 = sorted(rng.integers(-3, H + 3, 2) * SUB)
        else:                # fractional corners
            X0, X1 = sorted(rng.integers(-3 * SUB, (W + 3) * SUB, 2))
            Y0, Y1 = sorted(rng.integers(-3 * SUB, (H + 3) * SUB, 2))
        if X0 == X1 or Y0 == Y1:
            continue
        S, frags, culled, _ = _raster(_quad_tris(X0, Y0, X1, Y1, trial % 2, rng), W, H)
        want = _quad_count(int(X0), int(Y0), int(X1), int(Y1), W, H)
        assert int(S.sum()) == want
        assert frags == want, "diagonal double-covered or missed"
        assert culled == 0


@pytest.mark.parametrize("W,H", [(1, 1), (16, 16), (160, 128), (640, 512)])
def test_full_screen_quad(W, H):
    X0, Y0, X1, Y1 = -SUB // 2, -SUB // 2, W * SUB - SUB // 2, H * SUB - SUB // 2
    S, frags, _, _ = _raster(_quad_tris(X0, Y0, X1, Y1, 0, np.random.default_rng(0)), W, H)
    assert int(S.sum()) == W * H
    assert frags == W * H


def test_quad_edges_through_pixel_centres():
    # corners exactly on pixel centres (2,3)-(7,9): left/top included, right/bottom not
    W, H = 12, 12
    S, frags, _, _ = _raster(_quad_tris(2 * SUB, 3 * SUB, 7 * SUB, 9 * SUB, 1, np.random.default_rng(1)), W, H)
    want = np.zeros((H, W), np.uint8)
    want[3:9, 2:7] = 1
    assert np.array_equal(S, want)
    assert frags == 30


def _grid_tessellation(X0, Y0, X1, Y1, n, m, rng, jitter):
    xs = np.linspace(X0, X1, n + 1)
    ys = np.linspace(Y0, Y1, m + 1)
    P = {}
    for a in range(n + 1):
        for b in range(m + 1):
            x, y = xs[a], ys[b]
            if 0 < a < n:
                x += rng.uniform(-jitter, jitter)
            if 0 < b < m:
                y += rng.uniform(-jitter, jitter)
            P[a, b] = (int(round(x)), int(round(y)))
    tris = []
    for a in range(n):
        for b in range(m):
            p00, p10, p11, p01 = P[a, b], P[a + 1, b], P[a + 1, b + 1], P[a, b + 1]
            if rng.integers(2):
                tris += [(p00, p10, p11), (p00, p11, p01)]
            else:
                tris += [(p00, p10, p01), (p10, p11, p01)]
    return tris


@pytest.mark.parametrize("seed", range(8))
def test_watertight_grid_tessellation(seed):
    rng = np.random.default_rng(100 + seed)
    W, H = 48, 40
    X0, X1 = sorted(rng.integers(-2 * SUB, (W + 2) * SUB, 2))
    Y0, Y1 = sorted(rng.integers(-2 * SUB, (H + 2) * SUB, 2))
    n, m = rng.integers(1, 9, 2)
    jitter = 0.3 * min((X1 - X0) / n, (Y1 - Y0) / m)
    tris = _grid_tessellation(X0, Y0, X1, Y1, n, m, rng, jitter)
    S, frags, _, _ = _raster(tris, W, H)
    want = _quad_count(int(X0), int(Y0), int(X1), int(Y1), W, H)
    assert int(S.sum()) == want
    assert frags == want  # every covered pixel exactly once


@pytest.mark.parametrize("seed", range(8))
def test_watertight_fan(seed):
    rng = np.random.default_rng(200 + seed)
    W, H = 40, 40
    X0, Y0 = rng.integers(-SUB, 10 * SUB, 2)
    X1, Y1 = X0 + rng.integers(5 * SUB, 30 * SUB), Y0 + rng.integers(5 * SUB, 30 * SUB)
    # convex polygon = the quad's corners plus points on its sides, fanned from an interior point
    ring = [(X0, Y0)]
    for _ in range(rng.integers(0, 3)):
        ring.append((int(rng.integers(X0 + 1, X1)), Y0))
    ring.sort()
    ring.append((X1, Y0))
    right = [(X1, int(y)) for y in sorted(rng.integers(Y0 + 1, Y1, rng.integers(0, 3)))]
    ring += right + [(X1, Y1)]
    bottom = [(int(x), Y1) for x in sorted(rng.integers(X0 + 1, X1, rng.integers(0, 3)), reverse=True)]
    ring += bottom + [(X0, Y1)]
    left = [(X0, int(y)) for y in sorted(rng.integers(Y0 + 1, Y1, rng.integers(0, 3)), reverse=True)]
    ring += left
    ring = [r for i, r in enumerate(ring) if r != ring[i - 1]]
    c = (int(rng.integers(X0 + 1, X1)), int(rng.integers(Y0 + 1, Y1)))
    tris = [(c, ring[i], ring[(i + 1) % len(ring)]) for i in range(len(ring))]
    S, frags, _, _ = _raster(tris, W, H)
    want = _quad_count(int(X0), int(Y0), int(X1), int(Y1), W, H)
    assert int(S.sum()) == want
    assert frags == want


# ---------------------------------------------------------------------------
# Third implementation: exact rationals, top-left rule stated geometrically
# (a "top" edge is horizontal with the triangle below it; a "left" edge is
# non-horizontal with the triangle to its right).
# ---------------------------------------------------------------------------

def _orient(p, q, r):
    return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])


def _is_top_or_left(p, q, r):
    if p[1] == q[1]:
        return r[1] > p[1]  # y grows downwards: triangle below a top edge
    x_at = Fraction(p[0]) + Fraction(r[1] - p[1]) * Fraction(q[0] - p[0], q[1] - p[1])
    return r[0] > x_at


def _fraction_cover(tri, W, H):
    a, b, c = [(Fraction(x, SUB), Fraction(y, SUB)) for x, y in tri]
    area = _orient(a, b, c)
    S = np.zeros((H, W), np.uint8)
    if area == 0:
        return S
    edges = [(a, b, c), (b, c, a), (c, a, b)]
    for i in range(H):
        for j in range(W):
            P = (Fraction(j), Fraction(i))
            ok = True
            for p, q, r in edges:
                s = _orient(p, q, P) * (1 if area > 0 else -1)
                if s < 0 or (s == 0 and not _is_top_or_left(p, q, r)):
                    ok = False
                    break
            S[i, j] = ok
    return S


@pytest.mark.parametrize("seed", range(10))
def test_fraction_brute_force_tiny(seed):
    rng = np.random.default_rng(300 + seed)
    W, H = int(rng.integers(3, 13)), int(rng.integers(3, 13))
    for _ in range(25):
        mode = rng.integers(3)
        if mode == 0:   # on the pixel lattice: many centre-on-edge and vertex cases
            tri = [tuple(int(v) * SUB for v in rng.integers(-2, max(W, H) + 2, 2)) for _ in range(3)]
        elif mode == 1:  # half-pixel lattice
            tri = [tuple(int(v) * SUB // 2 for v in rng.integers(-4, 2 * max(W, H) + 4, 2)) for _ in range(3)]
        else:
            tri = [tuple(int(v) for v in rng.integers(-2 * SUB, (max(W, H) + 2) * SUB, 2)) for _ in range(3)]
        S, frags, _, _ = _raster([tuple(tri)], W, H)
        want = _fraction_cover(tri, W, H)
        assert np.array_equal(S, want), (tri, W, H)
        assert frags == int(want.sum())


def test_vertex_order_and_permutation_invariance():
    rng = np.random.default_rng(7)
    W, H = 30, 24
    tris = [tuple(tuple(int(v) for v in rng.integers(-SUB, 31 * SUB, 2)) for _ in range(3)) for _ in range(12)]
    S0, _, _, _ = _raster(tris, W, H)
    for perm in itertools.islice(itertools.permutations(range(3)), 6):
        t2 = [tuple(t[k] for k in perm) for t in tris]
        S1, _, _, _ = _raster(t2[::-1], W, H)
        assert np.array_equal(S0, S1)


def test_integer_pixel_translation_shifts_coverage():
    rng = np.random.default_rng(8)
    W, H = 40, 32
    tris = [tuple(tuple(int(v) for v in rng.integers(5 * SUB, 20 * SUB, 2)) for _ in range(3)) for _ in range(5)]
    S0, _, _, _ = _raster(tris, W, H)
    dj, di = 7, 4
    t2 = [tuple((x + dj * SUB, y + di * SUB) for x, y in t) for t in tris]
    S1, _, _, _ = _raster(t2, W, H)
    assert np.array_equal(S1[di:, dj:], S0[:H - di, :W - dj])
    assert S0[H - di:, :].sum() == 0 and S0[:, W - dj:].sum() == 0


def test_flagged_vertex_culls_triangle():
    pts = np.array([[0, 0], [10 * SUB, 0], [0, 10 * SUB]], np.int64)
    tris = np.array([[0, 1, 2]], np.int32)
    S, frags, culled, _ = oracle.raster(pts, np.array([0, 1, 0], np.uint8), tris, 16, 16)
    assert S.sum() == 0 and culled == 1


def test_area_bound_general_triangles():
    # |count - area| is at most the number of boundary-adjacent pixels (<= perimeter + 4)
    rng = np.random.default_rng(9)
    W, H = 64, 64
    for _ in range(50):
        tri = [tuple(int(v) for v in rng.integers(4 * SUB, 60 * SUB, 2)) for _ in range(3)]
        S, frags, _, _ = _raster([tuple(tri)], W, H)
        (x0, y0), (x1, y1), (x2, y2) = [(x / SUB, y / SUB) for x, y in tri]
        area = abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)) / 2
        per = math.dist((x0, y0), (x1, y1)) + math.dist((x1, y1), (x2, y2)) + math.dist((x2, y2), (x0, y0))
        assert abs(int(S.sum()) - area) <= per + 4


def test_counts_and_losses():
    rng = np.random.default_rng(10)
    S = (rng.random((20, 30)) < 0.4).astype(np.uint8)
    M = (rng.random((20, 30)) < 0.3).astype(np.uint8)
    s, m, I, x = oracle.counts(S, M)
    assert s == S.sum() and m == M.sum() and I == (S & M).sum()
    # MSE of binary images equals the XOR count (Eq. render_loss)
    assert x == ((S.astype(int) - M.astype(int)) ** 2).sum() == s + m - 2 * I
    l_xor = oracle.loss_from_counts(0, s, m, I)
    l_iou = oracle.loss_from_counts(1, s, m, I)
    l_app = oracle.loss_from_counts(2, s, m, I, lambda_app=0.5)
    assert l_xor == np.float32(x)
    assert l_iou == np.float32(1) - np.float32(I) / np.float32(s + m - I)
    assert abs(float(l_iou) - (1 - (S & M).sum() / (S | M).sum())) < 1e-6
    assert l_app == np.float32(x) + np.float32(0.5) * np.float32(abs(int(s) - int(m)))
    assert oracle.loss_from_counts(1, 0, 0, 0) == 0.0  # empty union: zero loss
