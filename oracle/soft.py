"""Soft silhouette loss and its gradient, FP64 (test infrastructure only).

The differentiable variant of the silhouette fitness: the paper renders its
silhouettes with a differentiable rasteriser (Sec. III-A.2) and compares them
with the mask in the MSE term of Eq. (render_loss); this module states the soft
form used here as a plain definition, pixel by pixel and triangle by triangle:

  d_t(p)  signed Euclidean distance (px) from pixel centre p = (j, i) to the
          boundary of projected triangle t, from the unsnapped projection:
          + inside (distance to the nearest edge line), - outside (distance to
          the nearest point of the triangle)
  a_t(p)  = sigmoid(d_t(p) / sigma), and 0 where d_t(p) < -cutoff * sigma
  S(p)    = 1 - prod_t (1 - a_t(p))        over every triangle of every link
  L       = sum_p (S(p) - M(p))^2          (the MSE term, Eq. render_loss)

with sigma = 1 px and cutoff = 14.  Triangles with a flagged vertex (behind
z_near or outside the guard band) and triangles of zero area are left out, as
in the binary renderer.  The products are kept in log form:
1 - a_t = exp(-softplus(d_t / sigma)).

The gradient follows the chain rule term by term:
  dL/dS(p) = 2 (S - M),  dS/da_t = prod_{t' != t} (1 - a_t'),  da/dd = a (1 - a) / sigma
so dL/dd_t(p) = 2 (S - M) (1 - S) sigmoid(d_t / sigma) / sigma, then through the
closest-feature geometry to the projected vertices (u, v), through the pinhole
projection to camera coordinates X, and through the kinematics to the state.
The last step uses the derivatives of the camera-from-frame transforms, taken
here by central differences of the oracle's own frame transforms (FP64, step
1e-6): X_v = T_f [v; 1] is linear in T_f, so dL/dtheta_k = sum_f <G_f, dT_f/dtheta_k>
with G_f = sum over the vertices of frame f of (dL/dX_v) [v; 1]^T.
"""
from __future__ import annotations

import numpy as np

from . import _flat_mesh, project

SIGMA = 1.0
CUTOFF = 14.0


def softplus(x):
    x = np.asarray(x, np.float64)
    return np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))


def sigmoid(x):
    x = np.asarray(x, np.float64)
    e = np.exp(-np.abs(x))
    return np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def _doubled_area(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def signed_distance(tri, px, py, grad: bool = False):
    """Signed distance from points (px, py) to the boundary of triangle tri
    (3 x 2, positively oriented).  With grad=True also returns the derivative
    with respect to the 6 vertex coordinates [x0 y0 x1 y1 x2 y2] (shape
    px.shape + (6,)).

    Edge k runs from vertex k to vertex k+1; E_k(p) = dx (py - y0) - dy (px - x0)
    is >= 0 on the inner side; h_k = E_k / |e_k| is the signed distance to the
    edge's line.  Inside (every E_k >= 0): d = min_k h_k.  Outside: d = -min_k
    dist(p, segment k), the segment distance being |E_k| / |e_k| when the foot
    of the perpendicular falls on the segment, else the distance to the nearer
    endpoint."""
    px = np.asarray(px, np.float64)
    py = np.asarray(py, np.float64)
    shape = px.shape
    h = np.empty((3,) + shape)
    seg = np.empty((3,) + shape)
    gh = np.zeros((3,) + shape + (6,))
    gs = np.zeros((3,) + shape + (6,))
    for k in range(3):
        k1 = (k + 1) % 3
        x0, y0 = tri[k]
        x1, y1 = tri[k1]
        dx, dy = x1 - x0, y1 - y0
        L2 = dx * dx + dy * dy
        L = np.sqrt(L2)
        E = dx * (py - y0) - dy * (px - x0)
        h[k] = E / L
        s = ((px - x0) * dx + (py - y0) * dy) / L2
        d0 = np.hypot(px - x0, py - y0)
        d1 = np.hypot(px - x1, py - y1)
        perp = (s > 0) & (s < 1)
        seg[k] = np.where(perp, np.abs(E) / L, np.where(s <= 0, d0, d1))
        if grad:
            # dE / d(x0, y0, x1, y1)
            dE = np.stack([y1 - py, px - x1, py - y0, -(px - x0)], axis=-1)
            dL = np.array([-dx, -dy, dx, dy]) / L
            dh = dE / L - (E / L2)[..., None] * dL  # d(E/L) = dE/L - E dL / L^2
            idx = [2 * k, 2 * k + 1, 2 * k1, 2 * k1 + 1]
            gh[k][..., idx] = dh
            sgn = np.sign(E)[..., None]
            g_perp = sgn * dh
            with np.errstate(invalid="ignore", divide="ignore"):
                g_v0 = np.stack([(x0 - px) / d0, (y0 - py) / d0], axis=-1)
                g_v1 = np.stack([(x1 - px) / d1, (y1 - py) / d1], axis=-1)
            g = np.zeros(shape + (6,))
            g[..., idx] = np.where(perp[..., None], g_perp, 0.0)
            end0 = ~perp & (s <= 0)
            end1 = ~perp & (s > 0)
            g[..., [2 * k, 2 * k + 1]] += np.where(end0[..., None], np.nan_to_num(g_v0), 0.0)
            g[..., [2 * k1, 2 * k1 + 1]] += np.where(end1[..., None], np.nan_to_num(g_v1), 0.0)
            gs[k] = g
    inside = (h >= 0).all(axis=0)
    kin = np.argmin(h, axis=0)
    kout = np.argmin(seg, axis=0)
    d = np.where(inside, np.take_along_axis(h, kin[None], 0)[0], -np.take_along_axis(seg, kout[None], 0)[0])
    if not grad:
        return d
    gi = np.take_along_axis(gh, kin[None, ..., None], 0)[0]
    go = -np.take_along_axis(gs, kout[None, ..., None], 0)[0]
    return d, np.where(inside[..., None], gi, go)


def _instrument_triangles(scene, state):
    """Per instrument: image-space vertex positions (u, v) [V, 2], flags,
    camera-frame positions X [V, 3] and the frame transforms."""
    K = scene.K
    out = []
    _, tris, vframe = _flat_mesh(scene)
    verts = np.concatenate([np.asarray(m.verts, np.float64) for m in scene.meshes])
    for b in range(scene.n_instruments):
        st = np.asarray(state, np.float64)[9 * b: 9 * b + 9]
        pr = project(scene, st)
        T = pr["T"]
        X = np.einsum("vij,vj->vi", T[vframe][:, :, :3], verts) + T[vframe][:, :, 3]
        uvimg = pr["uv"] + np.array([K.cx, K.cy])
        out.append(dict(uv=uvimg, off=pr["uv"], flag=pr["flag"], X=X, T=T, state=st))
    return out, tris, vframe, verts


def _windows(tri_list, W, H, sigma, cutoff):
    """For each drawable triangle (positively oriented, 3 x 2 image-space
    vertices): its index, the clipped pixel window of its bounding box grown by
    cutoff * sigma, and the pixel centres (px, py) of that window."""
    m = cutoff * sigma
    for n, tri in enumerate(tri_list):
        j0 = max(0, int(np.ceil(tri[:, 0].min() - m)))
        j1 = min(W - 1, int(np.floor(tri[:, 0].max() + m)))
        i0 = max(0, int(np.ceil(tri[:, 1].min() - m)))
        i1 = min(H - 1, int(np.floor(tri[:, 1].max() + m)))
        if j0 > j1 or i0 > i1:
            continue
        py, px = np.mgrid[i0:i1 + 1, j0:j1 + 1].astype(np.float64)
        yield n, (i0, i1, j0, j1), px, py


def soft_from_triangles(tri_list, W: int, H: int, sigma: float = SIGMA, cutoff: float = CUTOFF):
    """S [H, W] and the per-pixel softplus sum for image-space triangles
    (each 3 x 2, any orientation; zero-area triangles are left out)."""
    acc = np.zeros((H, W))
    tl = []
    for t in tri_list:
        t = np.asarray(t, np.float64)
        A = _doubled_area(*t)
        if A != 0:
            tl.append(t if A > 0 else t[[0, 2, 1]])
    for n, (i0, i1, j0, j1), px, py in _windows(tl, W, H, sigma, cutoff):
        d = signed_distance(tl[n], px, py)
        acc[i0:i1 + 1, j0:j1 + 1] += np.where(d >= -cutoff * sigma, softplus(d / sigma), 0.0)
    return 1.0 - np.exp(-acc), acc


def _drawable(scene, inst, tris):
    """(instrument, positively ordered vertex ids, image-space triangle) for every
    triangle without a flagged vertex and with nonzero area."""
    out = []
    for b, I in enumerate(inst):
        for t in tris:
            if I["flag"][t].any():
                continue
            A = _doubled_area(*I["uv"][t])
            if A == 0:
                continue
            ids = [t[0], t[1], t[2]] if A > 0 else [t[0], t[2], t[1]]
            out.append((b, ids, I["uv"][ids]))
    return out


def soft_render(scene, state, sigma: float = SIGMA, cutoff: float = CUTOFF):
    """S [H, W] (FP64) of one candidate and the per-pixel sum of softplus terms."""
    K = scene.K
    inst, tris, _, _ = _instrument_triangles(scene, state)
    return soft_from_triangles([tri for _, _, tri in _drawable(scene, inst, tris)], K.width, K.height, sigma,
                               cutoff)


def soft_loss(scene, state, mask, sigma: float = SIGMA, cutoff: float = CUTOFF) -> float:
    S, _ = soft_render(scene, state, sigma, cutoff)
    return float(((S - np.asarray(mask, np.float64)) ** 2).sum())


def soft_grad(scene, state, mask, sigma: float = SIGMA, cutoff: float = CUTOFF, fd_step: float = 1e-6):
    """(L, dL/dstate [d]) for one candidate."""
    K = scene.K
    M = np.asarray(mask, np.float64)
    S, _ = soft_render(scene, state, sigma, cutoff)
    L = float(((S - M) ** 2).sum())
    gS = 2.0 * (S - M) * (1.0 - S)  # dL/dd = gS * sigmoid(d / sigma) / sigma
    inst, tris, vframe, verts = _instrument_triangles(scene, state)
    guv = [np.zeros((verts.shape[0], 2)) for _ in inst]
    dr = _drawable(scene, inst, tris)
    for n, (i0, i1, j0, j1), px, py in _windows([tri for _, _, tri in dr], K.width, K.height, sigma, cutoff):
        b, ids, tri = dr[n]
        d, gd = signed_distance(tri, px, py, grad=True)
        keep = d >= -cutoff * sigma
        w = np.where(keep, gS[i0:i1 + 1, j0:j1 + 1] * sigmoid(d / sigma) / sigma, 0.0)
        g6 = (w[..., None] * gd).reshape(-1, 6).sum(axis=0)
        for k in range(3):
            guv[b][ids[k]] += g6[2 * k: 2 * k + 2]
    grad = np.zeros(9 * scene.n_instruments)
    for b, I in enumerate(inst):
        X, Z = I["X"], I["X"][:, 2]
        ok = I["flag"] == 0
        gu, gv = guv[b][:, 0], guv[b][:, 1]
        # u - cx = fx X / Z, v - cy = fy Y / Z
        gX = np.zeros_like(X)
        gX[ok, 0] = gu[ok] * K.fx / Z[ok]
        gX[ok, 1] = gv[ok] * K.fy / Z[ok]
        gX[ok, 2] = -(gu[ok] * I["off"][ok, 0] + gv[ok] * I["off"][ok, 1]) / Z[ok]
        vh = np.concatenate([verts, np.ones((verts.shape[0], 1))], axis=1)
        nF = I["T"].shape[0]
        G = np.zeros((nF, 3, 4))
        for f in range(nF):
            sel = vframe == f
            G[f] = gX[sel].T @ vh[sel]
        for k in range(9):
            e = np.zeros(9)
            e[k] = fd_step
            Tp = project(scene, I["state"] + e)["T"]
            Tm = project(scene, I["state"] - e)["T"]
            dT = (Tp - Tm) / (2 * fd_step)
            grad[9 * b + k] = float((G * dT).sum())
    return L, grad
