// Fitness of a CMA-ES population in one launch (arXiv 2603.11404, Sec. III-A.2):
//   S = R(K(Pi(T_r^c T_m^r(q) v_m))),  counts (s, I, m) of S against M_ref,
//   loss of Eq. render_loss / the 1 - IoU mask error of Sec. IV-B.
//
// Launch shape: one thread-block cluster of `cluster` CTAs per candidate.
//   prologue every CTA of the cluster (in the fused CMA-ES mode) samples the
//            candidate and composes its link transforms in double-float
//            arithmetic (redundantly: no CTA waits for another).
//   phase 1  every CTA projects its share of the vertices in compensated FP32
//            (double-float, error-free TwoSum/TwoProd), snapping them to 1/256 px
//            with round-half-even; the snapped vertices go to an L2-resident
//            scratch array.
//   phase 2  after a cluster barrier the warps of all CTAs take chunks of 32
//            triangles from a counter in CTA 0's shared memory until none
//            are left: integer setup (orientation, top-left bias, bbox), then
//            small triangles are rasterised by one thread each with int32
//            incremental edge functions, larger ones by a whole warp with
//            int64 edge functions and __ballot_sync coverage words.  Coverage
//            is OR-ed into the CTA's own full-image bitmap in shared memory.
//   phase 3  after a second cluster barrier CTA r ORs band r of all the
//            cluster's bitmaps through distributed shared memory, ANDs with
//            the observed mask, popcounts, and the cluster's counts meet in
//            CTA 0, which writes counts and loss.
// No silhouette image is written to global memory.
#include <cooperative_groups.h>

#include "cma_device.cuh"
#include "df.cuh"

namespace cg = cooperative_groups;

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

__device__ void compose_frames_warp(const ChainDev &ch, const CamDev &cam, const float *st, float *out,
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
// so that |e| < 2^28 over the bbox and a row fits one 64-bit word window.
// Each row collects its coverage most-significant-bit first (bits = 2 bits +
// sign), then one bit reversal puts pixel j0 at bit 0.
__device__ __forceinline__ void raster_small(const TriSetup &t, uint32_t *bm, int Wq)
{
    int r[3], cs[3], rs[3];
    long long Px = 256LL * t.j0, Py = 256LL * t.i0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int k1 = (k == 2) ? 0 : k + 1;
        int dx = t.x[k1] - t.x[k], dy = t.y[k1] - t.y[k];
        r[k] = (int)edge64(t, k, Px, Py);
        cs[k] = dy * 256;
        rs[k] = dx * 256;
    }
    const int jb = t.j0 & ~31;
    const int off = t.j0 - jb;
    const int nb = t.j1 - t.j0 + 1;  // 1..32
    uint32_t *row = bm + (size_t)t.i0 * Wq + (jb >> 5);
    for (int i = t.i0; i <= t.i1; ++i) {
        int a0 = r[0], a1 = r[1], a2 = r[2];
        uint32_t bits = 0u;
#pragma unroll 4
        for (int n = 0; n < nb; ++n) {
            bits = (bits << 1) | ((uint32_t)(~(a0 | a1 | a2)) >> 31);
            a0 -= cs[0];
            a1 -= cs[1];
            a2 -= cs[2];
        }
        if (bits) {
            unsigned long long m = (unsigned long long)(__brev(bits) >> (32 - nb)) << off;
            uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
            if (lo) atomicOr(row, lo);
            if (hi) atomicOr(row + 1, hi);
        }
        r[0] += rs[0];
        r[1] += rs[1];
        r[2] += rs[2];
        row += Wq;
    }
}

// One whole warp per triangle: lane l tests pixel 32 w + l of word w, int64 edges.
__device__ void raster_warp(const TriSetup &t, uint32_t *bm, int Wq, int lane)
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
__device__ void raster_serial(const TriSetup &t, uint32_t *bm, int Wq)
{
    for (int i = t.i0; i <= t.i1; ++i)
        for (int j = t.j0; j <= t.j1; ++j) {
            long long Px = 256LL * j, Py = 256LL * i;
            if ((edge64(t, 0, Px, Py) | edge64(t, 1, Px, Py) | edge64(t, 2, Px, Py)) >= 0)
                atomicOr(bm + (size_t)i * Wq + (j >> 5), 1u << (j & 31));
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

__device__ float keypoint_loss(const EvalArgs &a, const float *sM)
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

// Projected keypoints of given states (synthetic detections, diagnostics):
// one warp per state composes its frames and writes (u, v) of both keypoints
// of every instrument.
__global__ void k_project_keypoints(EvalArgs a, const float *states, int n, float *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nI = a.ch.n_inst, nF = a.ch.n_frames;
    float2 *scr = reinterpret_cast<float2 *>(smem);
    float *sM = reinterpret_cast<float *>(scr + nI * kComposeScratch);
    const int st = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (st >= n) return;
    if (warp < nI)
        compose_frames_warp(a.ch, a.cam, states + (size_t)st * a.d + 9 * warp, sM + warp * nF * 24,
                            scr + warp * kComposeScratch, lane);
    __syncthreads();
    if (threadIdx.x < 2 * nI) {
        const int b = threadIdx.x >> 1, k = threadIdx.x & 1;
        const float2 p = project_keypoint(sM + (b * nF + a.kp_frame[k]) * 24, a.kp_pt[k], a.cam);
        out[((size_t)st * nI + b) * 4 + 2 * k] = p.x;
        out[((size_t)st * nI + b) * 4 + 2 * k + 1] = p.y;
    }
}

cudaError_t launch_project_keypoints(const EvalArgs &a, const float *states, int n, float *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t smem = (size_t)a.ch.n_inst * (kComposeScratch * sizeof(float2) + a.ch.n_frames * 24 * sizeof(float));
    k_project_keypoints<<<n, 32 * a.ch.n_inst, smem, s>>>(a, states, n, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// The fused fitness kernel.
// ----------------------------------------------------------------------------
// One candidate c of one evaluation (all CTAs of the cluster call it together).
// mask_override replaces a.mask when not NULL (batched launches); fused_tell
// lets the last CTA of the launch run the CMA-ES update (single-instance mode).
// Programmatic dependent launch: consecutive fused generations are launched
// with programmatic stream serialisation, so the next generation's CTAs may be
// scheduled while this one is still running (its last CTA runs the update);
// they wait for this grid to complete, memory included, before reading
// anything.  Without that launch attribute both instructions do nothing.
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <bool kInlineFallback>
__device__ __forceinline__ void eval_candidate(const EvalArgs &a, int c, const uint32_t *mask_override,
                                               bool fused_tell, bool dependent_launch)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int K = (int)cluster.num_blocks();
    const uint32_t *maskp = mask_override ? mask_override : a.mask;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nI = a.ch.n_inst, nF = a.ch.n_frames;
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    const int nwords = H * Wq;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *scr = reinterpret_cast<float2 *>(smem);                           // [nI*kComposeScratch]
    uint32_t *bm = reinterpret_cast<uint32_t *>(scr + nI * kComposeScratch);  // [H*Wq]
    float *sM = reinterpret_cast<float *>(bm + ((nwords + 3) & ~3));          // [nI*nF*24]
    int *big = reinterpret_cast<int *>(sM + nI * nF * 24);                    // [kBigListCap]
    int *sacc = big + kBigListCap;  // [8]: s I m culled, big-list count, ticket counter, big-list overflow
    __shared__ int red[4][32];
    __shared__ float s_par[kMaxD];
    __shared__ float2 s_z[kMaxD];
    __shared__ int s_last;

    {  // the warps that do not compose frames clear the bitmap (16-byte stores)
        const int c0 = nwarp > nI ? 32 * nI : 0;
        uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
        for (int w = tid - c0; w >= 0 && w < (nwords + 3) >> 2; w += nthr - c0) bm4[w] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < 8) sacc[tid] = 0;
    // everything above touches only this CTA's shared memory; from here on the
    // launch reads what the previous generation wrote
    if (dependent_launch) griddep_wait();
    // ---- prologue: every CTA samples the candidate (fused CMA-ES mode; the
    //      draws are the same in every CTA and CTA 0 stores them) and composes
    //      its frames in double-float, so no CTA waits for another ----
    {
        const float *par = a.params + (size_t)c * a.d;
        if (a.cma_st) {
            if (warp == 0) {
                const bool owner = rank == 0;
                cma_sample_warp(*a.cma_k, a.cma_st, c, nullptr, owner ? a.cma_y : nullptr,
                                owner ? a.cma_z : nullptr, owner ? const_cast<float *>(a.params) : nullptr, s_par,
                                s_z, lane);
            }
            __syncthreads();
            par = s_par;
        }
        if (warp < nI)
            compose_frames_warp(a.ch, a.cam, par + 9 * warp, sM + warp * nF * 24, scr + warp * kComposeScratch,
                                lane);
    }
    __syncthreads();

    // ---- phase 1: project and snap this CTA's share of the vertices, two in flight ----
    const int gtid = rank * nthr + tid, gstride = K * nthr;
    int2 *snapc = a.snap + (size_t)c * nI * a.V;
    const int NV = nI * a.V;
    for (int idx0 = gtid; idx0 < NV; idx0 += 2 * gstride) {
        const int idx1 = idx0 + gstride;
        const bool has1 = idx1 < NV;
        int b0 = idx0 >= a.V, b1 = has1 ? (idx1 >= a.V) : b0;  // instrument (at most 2): no division
        float4 p0 = a.verts[idx0 - b0 * a.V];
        float4 p1 = has1 ? a.verts[idx1 - b1 * a.V] : p0;
        float2 uv0, uv1;
        int2 o0 = project_vertex(p0, sM + (b0 * nF + (int)p0.w) * 24, a.cam, uv0);
        int2 o1 = project_vertex(p1, sM + (b1 * nF + (int)p1.w) * 24, a.cam, uv1);
        snapc[idx0] = o0;
        if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx0] = o0;
        if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx0] = uv0;
        if (has1) {
            snapc[idx1] = o1;
            if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx1] = o1;
            if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx1] = uv1;
        }
    }
    cluster.sync();  // arrive.release / wait.acquire: the snapped vertices are visible cluster-wide

    // ---- phase 2: triangles -> this CTA's bitmap.  Warps of the whole cluster
    //      take chunks of 32 triangles (one per lane) from a counter in CTA 0's
    //      shared memory, so the cluster finishes together whatever the
    //      triangles cost; the bitmaps are OR-ed in phase 3, so which CTA draws a
    //      triangle does not change the result.  Three chunks are in flight:
    //      the next chunk's vertices, the one after's indices and a ticket ----
    int culled = 0;
    const int NT = nI * a.T;
    {
        int *ctr = cluster.map_shared_rank(&sacc[5], 0);
        auto ticket = [&]() {
            int v = 0;
            if (lane == 0) v = atomicAdd(ctr, 1);
            return __shfl_sync(0xffffffffu, v, 0);
        };
        // chunk being drawn (vertices loaded), next chunk (indices loaded), and
        // the one after (ticket taken)
        int cur = ticket(), nx1 = ticket(), nx2 = ticket();
        int t0 = cur * 32 + lane, t1 = nx1 * 32 + lane;
        int4 tri1 = make_int4(0, 0, 0, 0);
        int b1 = 0;
        int2 v0 = make_int2(0, 0), v1 = v0, v2 = v0;
        if (t0 < NT) {
            const int b0 = t0 >= a.T;  // instrument (at most 2): no division
            const int4 tri0 = a.tris[t0 - b0 * a.T];
            const int2 *sv = snapc + b0 * a.V;
            // written by other CTAs of the cluster in phase 1: read through L2
            v0 = __ldcg(sv + tri0.x);
            v1 = __ldcg(sv + tri0.y);
            v2 = __ldcg(sv + tri0.z);
        }
        if (t1 < NT) {
            b1 = t1 >= a.T;
            tri1 = a.tris[t1 - b1 * a.T];
        }
        while (cur * 32 < NT) {  // tickets of one warp increase: once past the end, done
            const int nx3 = ticket();
            int2 w0 = make_int2(0, 0), w1 = w0, w2 = w0;
            if (t1 < NT) {
                const int2 *svn = snapc + b1 * a.V;
                w0 = __ldcg(svn + tri1.x);
                w1 = __ldcg(svn + tri1.y);
                w2 = __ldcg(svn + tri1.z);
            }
            const int t2 = nx2 * 32 + lane;
            int4 tri2 = make_int4(0, 0, 0, 0);
            int b2 = 0;
            if (t2 < NT) {
                b2 = t2 >= a.T;
                tri2 = a.tris[t2 - b2 * a.T];
            }
            if (t0 < NT) {
                TriSetup t;
                const int st = tri_setup(v0, v1, v2, W, H, a.cull, t);
                if (st == 2) ++culled;
                if (st == 1) {
                    if (t.spanx < 32 * 256 && t.spany < 64 * 256) {
                        raster_small(t, bm, Wq);
                    } else {
                        // larger triangles wait for a whole warp.  If the list is
                        // full: the plain launch redraws every large triangle after
                        // the loop (raster code here would make its loop spill); the
                        // batched launch, compiled with more registers, draws the
                        // triangle in this lane
                        int slot = atomicAdd(&sacc[4], 1);
                        if (slot < kBigListCap) big[slot] = t0;
                        else if constexpr (kInlineFallback) raster_serial(t, bm, Wq);
                        else sacc[6] = 1;
                    }
                }
            }
            cur = nx1;
            t0 = t1;
            v0 = w0;
            v1 = w1;
            v2 = w2;
            nx1 = nx2;
            t1 = t2;
            tri1 = tri2;
            b1 = b2;
            nx2 = nx3;
        }
    }
    __syncthreads();
    const int nbig = min(sacc[4], kBigListCap);
    for (int e = warp; e < nbig; e += nwarp) {
        int tt = big[e];
        int b = tt >= a.T;
        int4 tri = a.tris[tt - b * a.T];
        const int2 *sv = snapc + b * a.V;
        TriSetup t;
        tri_setup(__ldcg(sv + tri.x), __ldcg(sv + tri.y), __ldcg(sv + tri.z), W, H, a.cull, t);
        raster_warp(t, bm, Wq, lane);
    }
    if (!kInlineFallback && sacc[6]) {  // the list overflowed: every large triangle of the candidate, a warp each (drawing twice is harmless)
        for (int base = warp * 32; base < NT; base += nwarp * 32) {
            const int tt = base + lane;
            bool large = false;
            TriSetup t;
            if (tt < NT) {
                const int b = tt >= a.T;
                const int4 tri = a.tris[tt - b * a.T];
                const int2 *sv = snapc + b * a.V;
                large = tri_setup(__ldcg(sv + tri.x), __ldcg(sv + tri.y), __ldcg(sv + tri.z), W, H, a.cull, t) == 1 &&
                        !(t.spanx < 32 * 256 && t.spany < 64 * 256);
            }
            for (unsigned mm = __ballot_sync(0xffffffffu, large); mm; mm &= mm - 1) {
                const int src = __ffs(mm) - 1, tu = __shfl_sync(0xffffffffu, tt, src);
                const int b = tu >= a.T;
                const int4 tri = a.tris[tu - b * a.T];
                const int2 *sv = snapc + b * a.V;
                TriSetup u;
                tri_setup(__ldcg(sv + tri.x), __ldcg(sv + tri.y), __ldcg(sv + tri.z), W, H, a.cull, u);
                raster_warp(u, bm, Wq, lane);
            }
        }
    }
    cluster.sync();

    // ---- phase 3: OR the cluster's bitmaps over this CTA's band, count ----
    const int per = (nwords + K - 1) / K;
    const int w0 = rank * per, w1 = min(nwords, w0 + per);
    const uint32_t *rbm[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rbm[q] = cluster.map_shared_rank(bm, q < K ? q : 0);
    int s = 0, I = 0, m = 0;
    for (int w = w0 + tid; w < w1; w += nthr) {
        uint32_t part[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) part[q] = (q < K) ? rbm[q][w] : 0u;
        uint32_t M = maskp[w];
        uint32_t S = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) S |= part[q];
        s += __popc(S);
        I += __popc(S & M);
        m += __popc(M);
        if (a.silhouette) a.silhouette[w] = S;
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        I += __shfl_xor_sync(0xffffffffu, I, o);
        m += __shfl_xor_sync(0xffffffffu, m, o);
        culled += __shfl_xor_sync(0xffffffffu, culled, o);
    }
    if (lane == 0) {
        red[0][warp] = s;
        red[1][warp] = I;
        red[2][warp] = m;
        red[3][warp] = culled;
    }
    __syncthreads();
    if (tid < 4) {
        int acc = 0;
        for (int w = 0; w < nwarp; ++w) acc += red[tid][w];
        atomicAdd(cluster.map_shared_rank(&sacc[tid], 0), acc);
    }
    cluster.sync();
    if (rank == 0 && tid == 0) {
        int S_ = sacc[0], I_ = sacc[1], M_ = sacc[2], C_ = sacc[3];
        if (a.counts) {
            a.counts[4 * c + 0] = S_;
            a.counts[4 * c + 1] = I_;
            a.counts[4 * c + 2] = M_;
            a.counts[4 * c + 3] = C_;
        }
        if (a.loss) {
            int x = S_ + M_ - 2 * I_;
            float L;
            if (a.loss_kind == TRK_LOSS_ONE_MINUS_IOU) {
                int U = S_ + M_ - I_;
                L = (U > 0) ? __fsub_rn(1.0f, __fdiv_rn((float)I_, (float)U)) : 0.0f;
            } else if (a.loss_kind == TRK_LOSS_MSE_APP) {
                L = __fadd_rn((float)x, __fmul_rn(a.lambda_app, (float)abs(S_ - M_)));
            } else {
                L = (float)x;
            }
            if (a.kp_obs && a.kp_lambda != 0.0f) L = __fadd_rn(L, keypoint_loss(a, sM));
            a.loss[c] = L;
        }
    }
    if (a.cma_st && fused_tell) {  // the last CTA to finish updates the search distribution
        if (tid == 0) {
            __threadfence();
            unsigned ticket = atomicAdd(a.cma_done, 1u);
            s_last = (ticket == gridDim.x * gridDim.y - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            TellSmem &S = *reinterpret_cast<TellSmem *>(smem);  // the cluster no longer reads this CTA's smem
            cma_tell_block(*a.cma_k, a.cma_st, a.cma_y, a.params, a.loss, S, tid, nthr);
            __syncthreads();
            if (a.cma_finish) cma_finish_frame(*a.cma_k, a.cma_st, a.cma_pose_out, tid, nthr);
            if (tid == 0) *a.cma_done = 0u;
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_eval(EvalArgs a)
{
    griddep_launch_dependents();
    eval_candidate<false>(a, blockIdx.y, nullptr, true, true);
}

// Persistent batched evaluation: a fixed grid of clusters pulls (instance,
// candidate) items from a queue (largest first) until it is empty.  CTA 0 of
// each cluster takes the ticket and the others read it through DSMEM, so the
// cluster stays in lockstep.  The CMA-ES update runs in a separate launch.
__global__ void __launch_bounds__(256, 3) k_eval_batch(const EvalArgs *descs, const uint32_t *const *masks,
                                                       const int2 *items, int n_items, unsigned *next_item)
{
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ int s_item;
    __shared__ __align__(16) EvalArgs s_args;  // this item's descriptor, read from shared memory
    for (;;) {
        if (cluster.block_rank() == 0 && threadIdx.x == 0) s_item = (int)atomicAdd(next_item, 1u);
        cluster.sync();
        const int it = *cluster.map_shared_rank(&s_item, 0);
        cluster.sync();  // every CTA has its ticket before CTA 0 takes the next
        if (it >= n_items) break;
        const int2 ic = items[it];
        const int4 *src = reinterpret_cast<const int4 *>(descs + ic.x);
        int4 *dst = reinterpret_cast<int4 *>(&s_args);
        for (int i = threadIdx.x; i < (int)(sizeof(EvalArgs) / 16); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        eval_candidate<true>(s_args, ic.y, masks ? masks[ic.x] : nullptr, false, false);
    }
}

cudaError_t launch_eval_batch(const EvalArgs *descs_dev, const uint32_t *const *masks_dev, const int2 *items_dev,
                              int n_items, unsigned *next_item_dev, const LaunchCfg &cfg, int n_clusters,
                              cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, n_clusters, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cfg.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_eval_batch, descs_dev, masks_dev, items_dev, n_items, next_item_dev);
}

cudaError_t prepare_eval_batch(size_t smem, int cluster, int threads, int *max_clusters)
{
    static size_t set_to = 0;
    cudaError_t e = cudaSuccess;
    if (smem > set_to) {
        e = cudaFuncSetAttribute(k_eval_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_to = smem;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cluster, 1, 1);
    lc.blockDim = dim3(threads, 1, 1);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, k_eval_batch, &lc);
}

size_t tell_smem_bytes() { return sizeof(TellSmem); }

size_t eval_smem_bytes(const EvalArgs &a)
{
    size_t nwords = (size_t)a.cam.H * a.cam.Wq;
    return (size_t)a.ch.n_inst * kComposeScratch * sizeof(float2) + ((nwords + 3) & ~(size_t)3) * 4 +
           (size_t)a.ch.n_inst * a.ch.n_frames * 24 * 4 + (size_t)kBigListCap * 4 + 8 * 4;
}

int eval_max_threads() { return 1024; }

cudaError_t prepare_eval(size_t smem)
{
    // The attribute is per function: raise it to the largest size any tracker needs.
    static size_t set_to = 0;
    if (smem <= set_to) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_to = smem;
    return e;
}

cudaError_t launch_eval(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s)
{
    if (a.lam == 0) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, a.lam, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cfg.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // fused generations follow each other: overlap the next one's launch with
    // this one's tail (see griddep_wait)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = a.cma_st ? 1 : 0;
    lc.attrs = attr;
    lc.numAttrs = 2;
    return cudaLaunchKernelEx(&lc, k_eval, a);
}

// ----------------------------------------------------------------------------
// Mask packing: one warp per 32-pixel word, coverage by __ballot_sync.
// ----------------------------------------------------------------------------
__global__ void k_pack_mask(const uint8_t *mask, uint32_t *packed, int W, int H, int Wq)
{
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (gw >= (long long)H * Wq) return;
    int i = (int)(gw / Wq), w = (int)(gw - (long long)i * Wq);
    int j = w * 32 + lane;
    bool on = (j < W) && mask[(size_t)i * W + j] != 0;
    unsigned b = __ballot_sync(0xffffffffu, on);
    if (lane == 0) packed[gw] = b;
}

cudaError_t launch_pack_mask(const uint8_t *mask, uint32_t *packed, int W, int H, int Wq, cudaStream_t s)
{
    long long threads = (long long)H * Wq * 32;
    int blocks = (int)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    k_pack_mask<<<blocks, 256, 0, s>>>(mask, packed, W, H, Wq);
    return cudaGetLastError();
}

}  // namespace trk
