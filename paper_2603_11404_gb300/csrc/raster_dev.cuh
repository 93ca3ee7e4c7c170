// Device building blocks of the fitness path shared by its kernels (the
// cluster-bitmap kernel in raster.cu and the binned pipeline in binned.cu):
// per-candidate kinematics in double-float arithmetic (Sec. III-A.2,
// III-A.3), compensated FP32 projection with the 1/256 px snap, integer
// triangle set-up and the top-left-rule raster primitives, and the keypoint
// term of Eq. kpts_loss.
#pragma once

#include "cma_device.cuh"
#include "df.cuh"

namespace trk {

// ----------------------------------------------------------------------------
// Per-candidate kinematics in double-float arithmetic (Sec. III-A.2, III-A.3)
// ----------------------------------------------------------------------------
__device__ __forceinline__ dfl dfc(float2 v) { return {v.x, v.y}; }

__device__ __forceinline__ dfl dot3(dfl a0, dfl b0, dfl a1, dfl b1, dfl a2, dfl b2)
{
    return df_add(df_add(df_mul(a0, b0), df_mul(a1, b1)), df_mul(a2, b2));
}

// Entry (i, j) of the elementary rotation about axis x/y/z (1/2/3; identity
// for TRK_AXIS_NONE) with sine s and cosine c.
__device__ __forceinline__ dfl rot_entry(int axis, dfl s, dfl c, int i, int j)
{
    const dfl one = df_from(1.0f), zero = df_from(0.0f);
    if (axis == TRK_AXIS_NONE) return i == j ? one : zero;
    const int a = axis - 1;  // the fixed coordinate
    if (i == a || j == a) return i == j ? one : zero;
    if (i == j) return c;
    // x: (1,2) = -s, (2,1) = s; y: (0,2) = s, (2,0) = -s; z: (0,1) = -s, (1,0) = s
    const bool neg = (axis == TRK_AXIS_Y) ? (i > j) : (i < j);
    return neg ? df_neg(s) : s;
}

// Projective rows of every frame for one instrument state, computed by one
// warp in double-float: rows (fx M0, fy M1, M2) of M = T_r^c T_f(q) with
// T_f = T_parent * [Rot(axis_f, coef_f q_joint) | offset_f] and q from the
// inverse cosine map q = lb + (ub-lb)/2 (1 - cos(pi (qh-lb)/(ub-lb))),
// written as hi/lo float pairs (24 floats per frame).  The pose rotation is
// axis-angle, R = cos t I + sin t [k]x + (1 - cos t) k k^T with t = |r|,
// k = r / t (I + [r]x when t < 1e-8), or look-at Ry(gamma) Rx(alpha) Rz(beta)
// (Sec. III-A.3).  The lanes run the same code on different data: one
// sine/cosine evaluation gives the three joint maps and the pose angles,
// a second one the joint rotations, then the chain products, level by level
// (frames at the same distance from the root in parallel).  The chain's root
// starts from G = diag(fx, fy, 1) [R | t], so each product down the chain
// yields the frame's scaled projective rows directly.
// scr: kComposeScratch float2 (a multiple of two, so what follows stays
// 16-byte aligned).
constexpr int kComposeScratch = 4 + 12 + kMaxFrames * 9 + kMaxFrames * 12;

static __device__ void compose_frames_warp(const ChainDev &ch, const CamDev &cam, const float *st, float *out,
                                    float2 *scr, int lane)
{
    float2 *qs = scr, *G = scr + 4, *Js = scr + 16, *Ts = scr + 16 + kMaxFrames * 9;
    const int nF = ch.n_frames;
    const bool lookat = ch.rot_param == TRK_ROT_LOOKAT;
    const dfl r0 = df_from(st[0]), r1 = df_from(st[1]), r2 = df_from(st[2]);
    const dfl t = lookat ? df_from(0.0f) : df_sqrt(dot3(r0, r0, r1, r1, r2, r2));
    // step 1: lanes 0-2 the joint maps' angles, lane 3 the pose angle t (or
    // the look-at angles gamma, alpha, beta on lanes 3-5)
    dfl arg = df_from(0.0f);
    if (lane < 3)
        arg = df_mul(df_sub(df_from(st[6 + lane]), dfc(ch.lb_df[lane])), dfc(ch.pi_over_range_df[lane]));
    else if (lane == 3)
        arg = lookat ? r2 : t;
    else if (lane == 4 && lookat)
        arg = r0;
    else if (lane == 5 && lookat)
        arg = r1;
    const dfl2 sc = df_sincos(arg);
    if (lane < 3) {
        const dfl q = df_fma(dfc(ch.half_range_df[lane]), df_sub(df_from(1.0f), sc.c), dfc(ch.lb_df[lane]));
        qs[lane] = make_float2(q.hi, q.lo);
    } else if (lane < 6) {  // pose sines and cosines, parked in the chain scratch
        Ts[2 * (lane - 3)] = make_float2(sc.s.hi, sc.s.lo);
        Ts[2 * (lane - 3) + 1] = make_float2(sc.c.hi, sc.c.lo);
    }
    __syncwarp();
    // step 2: joint rotations (lanes < nF) and the pose rotation (lanes 0-8)
    dfl ang = df_from(0.0f);
    if (lane < nF) ang = df_mul(dfc(ch.coef_df[lane]), dfc(qs[ch.joint[lane]]));
    const dfl2 fsc = df_sincos(ang);
    dfl Rv = df_from(0.0f);
    if (lane < 9) {
        const int i = lane / 3, j = lane - 3 * (lane / 3);
        if (lookat) {
            const dfl sg = dfc(Ts[0]), cg = dfc(Ts[1]), sa = dfc(Ts[2]), ca = dfc(Ts[3]), sb = dfc(Ts[4]),
                      cb = dfc(Ts[5]);
            dfl row[3];  // row i of Ry(gamma) Rx(alpha)
#pragma unroll
            for (int l = 0; l < 3; ++l)
                row[l] = dot3(rot_entry(TRK_AXIS_Y, sg, cg, i, 0), rot_entry(TRK_AXIS_X, sa, ca, 0, l),
                              rot_entry(TRK_AXIS_Y, sg, cg, i, 1), rot_entry(TRK_AXIS_X, sa, ca, 1, l),
                              rot_entry(TRK_AXIS_Y, sg, cg, i, 2), rot_entry(TRK_AXIS_X, sa, ca, 2, l));
            Rv = dot3(row[0], rot_entry(TRK_AXIS_Z, sb, cb, 0, j), row[1], rot_entry(TRK_AXIS_Z, sb, cb, 1, j),
                      row[2], rot_entry(TRK_AXIS_Z, sb, cb, 2, j));
        } else {
            const dfl r[3] = {r0, r1, r2};
            if (t.hi < 1e-8f) {
                // I + [r]x: (0,1) = -r2, (0,2) = r1, (1,0) = r2, (1,2) = -r0, (2,0) = -r1, (2,1) = r0
                const int m = 3 - i - j;
                const bool neg = ((i + 1) % 3) == j;
                Rv = i == j ? df_from(1.0f) : (neg ? df_neg(r[m]) : r[m]);
            } else {
                const dfl it = df_div(df_from(1.0f), t);
                const dfl s = dfc(Ts[0]), c = dfc(Ts[1]);
                const dfl ki = df_mul(r[i], it), kj = df_mul(r[j], it);
                dfl Kij = df_from(0.0f);
                if (i != j) {
                    const int m = 3 - i - j;
                    const bool neg = ((i + 1) % 3) == j;
                    const dfl km = df_mul(r[m], it);
                    Kij = neg ? df_neg(km) : km;
                }
                Rv = df_fma(df_sub(df_from(1.0f), c), df_mul(ki, kj), df_mul(s, Kij));
                if (i == j) Rv = df_add(Rv, c);
            }
        }
    }
    if (lane < nF) {
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const dfl v = rot_entry(ch.axis[lane], fsc.s, fsc.c, e / 3, e % 3);
            Js[9 * lane + e] = make_float2(v.hi, v.lo);
        }
    }
    // G = diag(fx, fy, 1) [R | t], row-major 3 x 4: lanes 0-8 the rotation
    // entries, lanes 9-11 the translation
    if (lane < 12) {
        const int i = lane < 9 ? lane / 3 : lane - 9;
        dfl g = lane < 9 ? Rv : df_from(st[3 + i]);
        if (i == 0) g = df_mul(g, dfc(cam.fx_df));
        if (i == 1) g = df_mul(g, dfc(cam.fy_df));
        G[lane < 9 ? 4 * i + (lane - 3 * i) : 4 * i + 3] = make_float2(g.hi, g.lo);
    }
    __syncwarp();
    // the chain, level by level (a frame's level is its distance from the root):
    // the frames of one level are independent, two at a time (12 lanes each,
    // lane = 4 i + j within a frame)
    int lvl = 0;
    if (lane < nF)
        for (int q = ch.parent[lane]; q >= 0; q = ch.parent[q]) ++lvl;
    int top = lvl;
    for (int o = 16; o; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
    for (int l = 0; l <= top; ++l) {
        for (unsigned fm = __ballot_sync(0xffffffffu, lane < nF && lvl == l); fm;) {
            const int fa = __ffs(fm) - 1;
            fm &= fm - 1;
            const int fb = fm ? __ffs(fm) - 1 : -1;
            if (fm) fm &= fm - 1;
            const int f = lane < 12 ? fa : (lane < 24 ? fb : -1);
            if (f >= 0) {
                const int e = lane < 12 ? lane : lane - 12, i = e >> 2, jj = e & 3;
                const float2 *Jf = Js + 9 * f;
                dfl L0 = jj < 3 ? dfc(Jf[jj]) : dfc(ch.offset_df[f][0]);
                dfl L1 = jj < 3 ? dfc(Jf[3 + jj]) : dfc(ch.offset_df[f][1]);
                dfl L2 = jj < 3 ? dfc(Jf[6 + jj]) : dfc(ch.offset_df[f][2]);
                const float2 *P = ch.parent[f] < 0 ? G : Ts + 12 * ch.parent[f];
                dfl v = dot3(dfc(P[4 * i]), L0, dfc(P[4 * i + 1]), L1, dfc(P[4 * i + 2]), L2);
                if (jj == 3) v = df_add(v, dfc(P[4 * i + 3]));
                Ts[12 * f + e] = make_float2(v.hi, v.lo);
            }
            __syncwarp();
        }
    }
    for (int e = lane; e < nF * 12; e += 32) {  // scaled rows of M_f, hi then lo
        const int f = e / 12, r = e - 12 * f;
        const float2 v = Ts[e];
        out[24 * f + r] = v.x;
        out[24 * f + 12 + r] = v.y;
    }
    __syncwarp();
}

// ----------------------------------------------------------------------------
// Compensated FP32 ("double-float") arithmetic: Knuth's TwoSum and the
// FMA-based TwoProd give exact rounding errors; explicit _rn intrinsics keep
// the compiler from contracting them.
// ----------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (hi + lo) . (x, y, z, 1)
__device__ __forceinline__ DF df_affine(const float *h, const float *l, float x, float y, float z)
{
    float p0, e0, p1, e1, p2, e2, s, t0, t1, t2;
    two_prod(h[0], x, p0, e0);
    two_prod(h[1], y, p1, e1);
    two_prod(h[2], z, p2, e2);
    two_sum(p0, p1, s, t0);
    two_sum(s, p2, s, t1);
    two_sum(s, h[3], s, t2);
    float err = __fadd_rn(__fadd_rn(t0, t1), __fadd_rn(t2, e0));
    err = __fadd_rn(err, __fadd_rn(e1, e2));
    err = __fadd_rn(err, __fmaf_rn(l[0], x, __fmaf_rn(l[1], y, __fmaf_rn(l[2], z, l[3]))));
    DF r;
    two_sum(s, err, r.hi, r.lo);
    return r;
}

// a / b given rb = 1/b.hi (approximate): one correction step from the exact residual.
__device__ __forceinline__ DF df_div(DF a, DF b, float rb)
{
    float q1 = __fmul_rn(a.hi, rb);
    float p, e;
    two_prod(q1, b.hi, p, e);
    float r = __fsub_rn(__fsub_rn(a.hi, p), e);
    r = __fadd_rn(r, __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
    float q2 = __fmul_rn(r, rb);
    DF o;
    two_sum(q1, q2, o.hi, o.lo);
    return o;
}

// Round-half-even of 256 (hi + lo), exact for |256 hi| < 2^22 (the guard band).
__device__ __forceinline__ int snap256(DF u)
{
    float a = __fmul_rn(u.hi, 256.0f);
    float b = __fmul_rn(u.lo, 256.0f);
    float n = rintf(a);
    float d = __fsub_rn(a, n);
    if (d == 0.5f && b > 0.0f) n = __fadd_rn(n, 1.0f);
    else if (d == -0.5f && b < 0.0f) n = __fsub_rn(n, 1.0f);
    return (int)n;
}

// ----------------------------------------------------------------------------
// Triangle setup shared by the raster paths.
// ----------------------------------------------------------------------------
struct TriSetup {
    int x[3], y[3];       // snapped vertices, positive orientation
    int j0, j1, i0, i1;   // pixel bbox clamped to the image
    int spanx, spany;     // vertex bbox extent in 1/256 px
};

// Returns 0 = nothing to draw, 1 = draw, 2 = culled for a flagged vertex.
// The clipped pixel bounding box is tested first: most triangles of a fine
// mesh contain no pixel centre and leave before the orientation test.
__device__ __forceinline__ int tri_setup(int2 a, int2 b, int2 c, int W, int H, int cull, TriSetup &t)
{
    if (a.x == kSnapFlag || b.x == kSnapFlag || c.x == kSnapFlag) return 2;
    int xmn = min(a.x, min(b.x, c.x)), xmx = max(a.x, max(b.x, c.x));
    int ymn = min(a.y, min(b.y, c.y)), ymx = max(a.y, max(b.y, c.y));
    t.j0 = max(0, (xmn + 255) >> 8);   // ceil(x / 256)
    t.j1 = min(W - 1, xmx >> 8);       // floor(x / 256)
    t.i0 = max(0, (ymn + 255) >> 8);
    t.i1 = min(H - 1, ymx >> 8);
    if (t.j0 > t.j1 || t.i0 > t.i1) return 0;
    t.spanx = xmx - xmn;
    t.spany = ymx - ymn;
    long long A;
    if (t.spanx < (1 << 15) && t.spany < (1 << 15)) {  // |products| < 2^30: int32 is exact
        A = (long long)((b.x - a.x) * (c.y - a.y) - (c.x - a.x) * (b.y - a.y));
    } else {
        A = (long long)(b.x - a.x) * (long long)(c.y - a.y) - (long long)(c.x - a.x) * (long long)(b.y - a.y);
    }
    if (A == 0) return 0;
    if (cull && A > 0) return 0;
    if (A < 0) {
        int2 tmp = b;
        b = c;
        c = tmp;
    }
    t.x[0] = a.x; t.y[0] = a.y;
    t.x[1] = b.x; t.y[1] = b.y;
    t.x[2] = c.x; t.y[2] = c.y;
    return 1;
}

// Edge k runs from vertex k to vertex k+1.  e_k(j, i) = dx (256 i - y_k)
// - dy (256 j - x_k) - bias_k, bias 0 on top-left edges (dy < 0, or dy == 0 and
// dx > 0) and 1 otherwise, so a pixel is covered iff every e_k >= 0.
__device__ __forceinline__ long long edge64(const TriSetup &t, int k, long long Px, long long Py)
{
    int k1 = (k == 2) ? 0 : k + 1;
    long long dx = t.x[k1] - t.x[k], dy = t.y[k1] - t.y[k];
    int bias = (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1;
    return dx * (Py - t.y[k]) - dy * (Px - t.x[k]) - bias;
}

// One thread, int32 incremental edges.  Requires spanx < 32 px and spany < 64 px
// so that |e| < 2^28 over the bbox (also at its corner, so the start values
// are exact in int32) and a row fits one 64-bit word window.  Each row
// collects its coverage most-significant-bit first (a funnel shift per
// pixel), then one bit reversal puts pixel j0 at bit 0.
// `row` points at the bitmap word holding pixel (t.i0, t.j0 & ~31); rows are
// `stride` words apart.
__device__ __forceinline__ void raster_small_at(const TriSetup &t, uint32_t *row, int stride)
{
    int r[3], cs[3], rs[3];
    const int Px = 256 * t.j0, Py = 256 * t.i0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k == 2) ? 0 : k + 1;
        const int dx = t.x[k1] - t.x[k], dy = t.y[k1] - t.y[k];
        const int bias = (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1;
        r[k] = dx * (Py - t.y[k]) - dy * (Px - t.x[k]) - bias;
        cs[k] = dy * 256;
        rs[k] = dx * 256;
    }
    const int jb = t.j0 & ~31;
    const int off = t.j0 - jb;
    const int nb = t.j1 - t.j0 + 1;  // 1..32
    const bool one_word = off + nb <= 32;
    for (int i = t.i0; i <= t.i1; ++i) {
        int a0 = r[0], a1 = r[1], a2 = r[2];
        uint32_t bits = 0u;
#pragma unroll 4
        for (int n = 0; n < nb; ++n) {
            bits = __funnelshift_l((uint32_t)(~(a0 | a1 | a2)), bits, 1);  // (bits << 1) | covered
            a0 -= cs[0];
            a1 -= cs[1];
            a2 -= cs[2];
        }
        if (bits) {
            const uint32_t rb = __brev(bits) >> (32 - nb);  // pixel j0 at bit 0
            if (one_word) {
                atomicOr(row, rb << off);
            } else {  // off >= 1 here
                const uint32_t lo = rb << off, hi = rb >> (32 - off);
                if (lo) atomicOr(row, lo);
                if (hi) atomicOr(row + 1, hi);
            }
        }
        r[0] += rs[0];
        r[1] += rs[1];
        r[2] += rs[2];
        row += stride;
    }
}

__device__ __forceinline__ void raster_small(const TriSetup &t, uint32_t *bm, int Wq)
{
    raster_small_at(t, bm + (size_t)t.i0 * Wq + ((t.j0 & ~31) >> 5), Wq);
}

// One whole warp per triangle: lane l tests pixel 32 w + l of word w, int64 edges.
static __device__ void raster_warp(const TriSetup &t, uint32_t *bm, int Wq, int lane)
{
    for (int i = t.i0; i <= t.i1; ++i) {
        long long Py = 256LL * i;
        for (int w = t.j0 >> 5; w <= (t.j1 >> 5); ++w) {
            int j = (w << 5) + lane;
            bool in = (j >= t.j0) && (j <= t.j1);
            if (in) {
                long long Px = 256LL * j;
                long long e = edge64(t, 0, Px, Py) | edge64(t, 1, Px, Py) | edge64(t, 2, Px, Py);
                in = e >= 0;
            }
            unsigned m = __ballot_sync(0xffffffffu, in);
            if (lane == 0 && m) atomicOr(bm + (size_t)i * Wq + w, m);
        }
    }
}

// One thread, int64, any size: the batched kernel's fallback when a CTA's
// deferred list is full.
static __device__ void raster_serial(const TriSetup &t, uint32_t *bm, int Wq)
{
    for (int i = t.i0; i <= t.i1; ++i)
        for (int j = t.j0; j <= t.j1; ++j) {
            long long Px = 256LL * j, Py = 256LL * i;
            if ((edge64(t, 0, Px, Py) | edge64(t, 1, Px, Py) | edge64(t, 2, Px, Py)) >= 0)
                atomicOr(bm + (size_t)i * Wq + (j >> 5), 1u << (j & 31));
        }
}

// ----------------------------------------------------------------------------
// Quadrilaterals: two mesh triangles T1 = (a, b, c) and T2 = (a, c, d) that share
// the edge a-c.  The top-left rule covers a pixel centre p exactly when the
// point p + (e, e^2), e -> 0+, lies strictly inside the triangle (for a
// non-horizontal edge the x shift decides the side, for a horizontal one the y
// shift).  That point never lies on the diagonal a-c, and when both triangles
// have the same orientation and (a, b, c, d) is strictly convex, the open
// quadrilateral minus the diagonal is the union of the two open triangles.  So
// the pixels of the quadrilateral under the same rule on its four edges are
// exactly the union of the two triangles' pixels: one set-up and one pass over
// one bounding box instead of two.  Anything else (a fold at a silhouette edge,
// a non-convex or degenerate pair, a flagged vertex) is drawn as two triangles.
// ----------------------------------------------------------------------------
struct QuadSetup {
    int x[4], y[4];       // snapped corners, positive orientation
    int j0, j1, i0, i1;   // pixel bbox clamped to the image
    int spanx, spany;     // corner bbox extent in 1/256 px
};

// Twice the signed area of (p, q, r); exact in int32 when every coordinate
// difference is below 2^15.
__device__ __forceinline__ long long orient2(int2 p, int2 q, int2 r, bool narrow)
{
    if (narrow) return (long long)((q.x - p.x) * (r.y - p.y) - (r.x - p.x) * (q.y - p.y));
    return (long long)(q.x - p.x) * (long long)(r.y - p.y) - (long long)(r.x - p.x) * (long long)(q.y - p.y);
}

// Returns 0 = nothing to draw (no pixel centre in the corners' clipped box, or
// both triangles culled as back faces), 1 = draw the quadrilateral, 3 = draw the
// two triangles separately (tri_setup on each; it also counts flagged ones).
__device__ __forceinline__ int quad_setup(int2 a, int2 b, int2 c, int2 d, int W, int H, int cull, QuadSetup &q)
{
    if (a.x == kSnapFlag || b.x == kSnapFlag || c.x == kSnapFlag || d.x == kSnapFlag) return 3;
    const int xmn = min(min(a.x, b.x), min(c.x, d.x)), xmx = max(max(a.x, b.x), max(c.x, d.x));
    const int ymn = min(min(a.y, b.y), min(c.y, d.y)), ymx = max(max(a.y, b.y), max(c.y, d.y));
    // each triangle's box lies inside this one: an empty box leaves both empty
    q.j0 = max(0, (xmn + 255) >> 8);
    q.j1 = min(W - 1, xmx >> 8);
    q.i0 = max(0, (ymn + 255) >> 8);
    q.i1 = min(H - 1, ymx >> 8);
    if (q.j0 > q.j1 || q.i0 > q.i1) return 0;
    q.spanx = xmx - xmn;
    q.spany = ymx - ymn;
    const bool narrow = q.spanx < (1 << 15) && q.spany < (1 << 15);
    const long long A1 = orient2(a, b, c, narrow), A2 = orient2(a, c, d, narrow);
    const long long Da = orient2(b, d, a, narrow), Dc = orient2(b, d, c, narrow);
    // same non-zero orientation, and a, c strictly on opposite sides of b-d
    const bool convex = ((A1 > 0 && A2 > 0) || (A1 < 0 && A2 < 0)) && ((Da > 0 && Dc < 0) || (Da < 0 && Dc > 0));
    if (!convex) return 3;
    if (cull && A1 > 0) return 0;
    if (A1 < 0) {  // reverse the corner order: positive orientation
        int2 t = b;
        b = d;
        d = t;
    }
    q.x[0] = a.x; q.y[0] = a.y;
    q.x[1] = b.x; q.y[1] = b.y;
    q.x[2] = c.x; q.y[2] = c.y;
    q.x[3] = d.x; q.y[3] = d.y;
    return 1;
}

// One thread, four int32 incremental edge functions (edge k from corner k to
// corner k+1, the top-left bias as in raster_small_at).  The same bounds as the
// triangle form: spanx < 32 px, spany < 64 px.
__device__ __forceinline__ void raster_quad_small(const QuadSetup &q, uint32_t *bm, int Wq)
{
    int r[4], cs[4], rs[4];
    const int Px = 256 * q.j0, Py = 256 * q.i0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        const int dx = q.x[k1] - q.x[k], dy = q.y[k1] - q.y[k];
        const int bias = (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1;
        r[k] = dx * (Py - q.y[k]) - dy * (Px - q.x[k]) - bias;
        cs[k] = dy * 256;
        rs[k] = dx * 256;
    }
    const int jb = q.j0 & ~31;
    const int off = q.j0 - jb;
    const int nb = q.j1 - q.j0 + 1;  // 1..32
    const bool one_word = off + nb <= 32;
    uint32_t *row = bm + (size_t)q.i0 * Wq + (jb >> 5);
    for (int i = q.i0; i <= q.i1; ++i) {
        int a0 = r[0], a1 = r[1], a2 = r[2], a3 = r[3];
        uint32_t bits = 0u;
#pragma unroll 4
        for (int n = 0; n < nb; ++n) {
            bits = __funnelshift_l((uint32_t)(~(a0 | a1 | a2 | a3)), bits, 1);  // (bits << 1) | covered
            a0 -= cs[0];
            a1 -= cs[1];
            a2 -= cs[2];
            a3 -= cs[3];
        }
        if (bits) {
            const uint32_t rb = __brev(bits) >> (32 - nb);  // pixel j0 at bit 0
            if (one_word) {
                atomicOr(row, rb << off);
            } else {
                const uint32_t lo = rb << off, hi = rb >> (32 - off);
                if (lo) atomicOr(row, lo);
                if (hi) atomicOr(row + 1, hi);
            }
        }
        r[0] += rs[0];
        r[1] += rs[1];
        r[2] += rs[2];
        r[3] += rs[3];
        row += Wq;
    }
}

// Camera-frame position of one vertex from its frame's projective rows (hi/lo
// pairs), perspective division and snap: int2 (U, V) in 1/256 px, or the flag
// value when the vertex is behind z_near or outside the guard band; uv gets
// the unsnapped offsets from the principal point.
__device__ __forceinline__ int2 project_vertex(float4 p, const float *Mh, const CamDev &cam, float2 &uv)
{
    DF X = df_affine(Mh + 0, Mh + 12, p.x, p.y, p.z);
    DF Y = df_affine(Mh + 4, Mh + 16, p.x, p.y, p.z);
    DF Z = df_affine(Mh + 8, Mh + 20, p.x, p.y, p.z);
    int2 o = make_int2(kSnapFlag, kSnapFlag);
    uv = make_float2(0.f, 0.f);
    if (Z.hi >= (float)cam.z_near) {
        float rz = __frcp_rn(Z.hi);
        DF u = df_div(X, Z, rz), w = df_div(Y, Z, rz);
        uv = make_float2(__fadd_rn(u.hi, u.lo), __fadd_rn(w.hi, w.lo));
        const float guard = (float)cam.guard;
        if (fabsf(u.hi) <= guard && fabsf(w.hi) <= guard)
            o = make_int2(snap256(u) + cam.cx256, snap256(w) + cam.cy256);
    }
    return o;
}

// ----------------------------------------------------------------------------
// Keypoint term (Eq. kpts_loss): the two keypoints of each instrument (the jaw
// tips) projected with the candidate's frames, compared with the detections
// under the better of the two assignments, plus their means, each distance
// reduced by the threshold tau and clipped at zero; summed over the
// instruments whose detection is valid (exactly two keypoints found), times
// lambda_kpts.  FP32 from the double-float frame rows.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float2 project_keypoint(const float *M, const float *pt, const CamDev &cam)
{
    // rows (fx M0, fy M1, M2) as hi/lo pairs: M[r] hi, M[12 + r] lo, r = 4 i + j
    float X[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float acc = M[4 * i + 3] + M[12 + 4 * i + 3];
#pragma unroll
        for (int j = 0; j < 3; ++j) acc = fmaf(M[4 * i + j] + M[12 + 4 * i + j], pt[j], acc);
        X[i] = acc;
    }
    return make_float2(X[0] / X[2] + cam.cx256 * (1.0f / 256.0f), X[1] / X[2] + cam.cy256 * (1.0f / 256.0f));
}

__device__ __forceinline__ float pos_part(float x) { return fmaxf(x, 0.0f); }

static __device__ float keypoint_loss(const EvalArgs &a, const float *sM)
{
    const int nF = a.ch.n_frames;
    float total = 0.0f;
    for (int b = 0; b < a.ch.n_inst; ++b) {
        const float *o = a.kp_obs + 5 * b;
        if (o[4] == 0.0f) continue;
        const float2 p0 = project_keypoint(sM + (b * nF + a.kp_frame[0]) * 24, a.kp_pt[0], a.cam);
        const float2 p1 = project_keypoint(sM + (b * nF + a.kp_frame[1]) * 24, a.kp_pt[1], a.cam);
        const float tau = a.kp_tau;
        const float same = pos_part(hypotf(o[0] - p0.x, o[1] - p0.y) - tau) + pos_part(hypotf(o[2] - p1.x, o[3] - p1.y) - tau);
        const float swap = pos_part(hypotf(o[0] - p1.x, o[1] - p1.y) - tau) + pos_part(hypotf(o[2] - p0.x, o[3] - p0.y) - tau);
        const float mean = pos_part(hypotf(0.5f * (o[0] + o[2]) - 0.5f * (p0.x + p1.x), 0.5f * (o[1] + o[3]) - 0.5f * (p0.y + p1.y)) - tau);
        total += fminf(same, swap) + mean;
    }
    return a.kp_lambda * total;
}

// A candidate's state with a NaN or an infinity: its projection flags every
// vertex; report it in the device error word (one warp per CTA calls this).
__device__ __forceinline__ void check_state_finite(const float *st, int d, unsigned *err, int lane)
{
    const bool bad = lane < d && !isfinite(st[lane]);
    if (__ballot_sync(0xffffffffu, bad) && lane == 0 && err) atomicOr(err, TRK_DEVERR_NONFINITE);
}

// Programmatic dependent launch: kernels that follow each other on a stream
// are launched with programmatic stream serialisation, so the next kernel's
// CTAs may be scheduled while this one is still running; they wait for this
// grid to complete, memory included, before reading anything it writes.
// Without that launch attribute both instructions do nothing.
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace trk
