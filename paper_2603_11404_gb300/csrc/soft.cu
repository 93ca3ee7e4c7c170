// Soft (differentiable) silhouette loss and its gradient: soft_eval and
// soft_refine in include/tracker.h.
//
// The soft form of the fitness (the paper fits with a differentiable
// renderer, Sec. III-A.2, and the MSE term of Eq. render_loss):
//   d_t(p)  signed distance (px) from pixel centre p to the boundary of
//           projected triangle t (+ inside, - outside), unsnapped coordinates
//   a_t(p)  sigmoid(d_t(p) / sigma), 0 where d_t(p) < -14 sigma
//   S(p)    1 - prod_t (1 - a_t(p)) = 1 - exp(-sum_t softplus(d_t(p) / sigma))
//   L       sum_p (S(p) - M(p))^2
// and dL/dd_t(p) = 2 (S - M) (1 - S) sigmoid(d_t / sigma) / sigma, taken back
// through the closest boundary feature to the projected vertices, through the
// pinhole to camera coordinates and through the kinematics to the state.
// Everything is FP32.
//
// Launches per call (one row of kernels per population):
//   k_soft_project  per (candidate, instrument): kinematics with the nine
//                   state tangents carried along (forward mode), vertex
//                   projection, screen box of the instrument
//   k_soft_tribox   per (candidate, triangle): window of influence (bounding
//                   box grown by 14 sigma) clipped to the image, and the union
//                   of the windows of every chunk of 256 triangles
//   k_soft_tile     per (candidate, 16x16 tile): pass 1 sums the softplus
//                   terms of every triangle whose window meets the tile into
//                   the tile's pixels and adds the tile's squared error to the
//                   loss; with a gradient, pass 2 recomputes the same pairs
//                   and scatters dL/d(u, v) to the vertices.  Nothing per pixel
//                   leaves the tile: the backward recomputes instead of storing.
//   k_soft_reduce   per (candidate, instrument): dL/dX per vertex, reduced per
//                   kinematic frame to a 3x4 matrix G_f, contracted with the
//                   frame tangents dT_f/dtheta_k; writes loss and gradient.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace trk {

constexpr float kSoftCutoff = 14.0f;   // in units of sigma
constexpr int kTile = 16;              // tile edge (px): one pixel per thread
constexpr int kSoftThreads = 256;
constexpr int kChunk = 256;            // triangles staged per pass
// Gradient sums are accumulated in 64-bit fixed point, exact and so independent
// of the order of the (atomic) additions: dL/d(u, v) per vertex in units of
// 2^-32 (|sum| < 2^31), the per-frame G_f in units of 2^-24 (|sum| < 2^39).
constexpr double kGvScale = 4294967296.0;
constexpr double kGScale = 16777216.0;
__device__ __forceinline__ long long to_fixed(float x, double scale) { return __double2ll_rn((double)x * scale); }

// ---------------------------------------------------------------------------
// Forward-mode kinematics: every lane carries the values and one tangent
// direction (lane k+1: d/dtheta_k, lane 0: none).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mul34(const float *A, const float *B, float *C)  // [R|t] * [R|t]
{
    float T[12];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float acc = (j == 3) ? A[4 * i + 3] : 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = fmaf(A[4 * i + k], B[4 * k + j], acc);
            T[4 * i + j] = acc;
        }
#pragma unroll
    for (int e = 0; e < 12; ++e) C[e] = T[e];
}

// Derivative of the product C = A B of two [R|t] transforms:
// dC_R = dA_R B_R + A_R dB_R, dC_t = dA_R B_t + A_R dB_t + dA_t.
__device__ __forceinline__ void dmul34(const float *dA, const float *B, const float *A, const float *dB, float *dC)
{
    float T[12];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float acc = (j == 3) ? dA[4 * i + 3] : 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = fmaf(dA[4 * i + k], B[4 * k + j], fmaf(A[4 * i + k], dB[4 * k + j], acc));
            T[4 * i + j] = acc;
        }
#pragma unroll
    for (int e = 0; e < 12; ++e) dC[e] = T[e];
}

// Elementary rotation about axis 1/2/3 (x/y/z) and its derivative by the angle.
__device__ __forceinline__ void rot_axis(int axis, float ang, float *R, float *dR)
{
    float s, c;
    sincosf(ang, &s, &c);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        R[e] = (e % 4 == 0) ? 1.0f : 0.0f;
        dR[e] = 0.0f;
    }
    if (axis == 1) {
        R[4] = c; R[5] = -s; R[7] = s; R[8] = c;
        dR[4] = -s; dR[5] = -c; dR[7] = c; dR[8] = -s;
    } else if (axis == 2) {
        R[0] = c; R[2] = s; R[6] = -s; R[8] = c;
        dR[0] = -s; dR[2] = c; dR[6] = -c; dR[8] = -s;
    } else if (axis == 3) {
        R[0] = c; R[1] = -s; R[3] = s; R[4] = c;
        dR[0] = -s; dR[1] = -c; dR[3] = c; dR[4] = -s;
    }
}

__device__ __forceinline__ void mul33(const float *A, const float *B, float *C)
{
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = fmaf(A[3 * i + k], B[3 * k + j], acc);
            T[3 * i + j] = acc;
        }
#pragma unroll
    for (int e = 0; e < 9; ++e) C[e] = T[e];
}

// Rotation of the state and its derivative along r_dir (dir < 0: none).
// Axis-angle: Rodrigues R = I + s K + c1 K^2 (t = |r|, k = r / t, s = sin t,
// c1 = 1 - cos t, K = [k]x), differentiated term by term; below t = 1e-4 the
// second-order series I + [r]x + [r]x^2 / 2.  Look-at: Ry(g) Rx(a) Rz(b).
__device__ void rotation_tangent(int rot_param, const float r[3], int dir, float *R, float *dR)
{
    if (rot_param == TRK_ROT_LOOKAT) {
        float Ry[9], dRy[9], Rx[9], dRx[9], Rz[9], dRz[9], T[9];
        rot_axis(2, r[2], Ry, dRy);
        rot_axis(1, r[0], Rx, dRx);
        rot_axis(3, r[1], Rz, dRz);
        mul33(Ry, Rx, T);
        mul33(T, Rz, R);
        if (dir == 0) { mul33(Ry, dRx, T); mul33(T, Rz, dR); }
        else if (dir == 1) { mul33(Ry, Rx, T); mul33(T, dRz, dR); }
        else if (dir == 2) { mul33(dRy, Rx, T); mul33(T, Rz, dR); }
        else for (int e = 0; e < 9; ++e) dR[e] = 0.0f;
        return;
    }
    const float e0 = dir == 0 ? 1.0f : 0.0f, e1 = dir == 1 ? 1.0f : 0.0f, e2 = dir == 2 ? 1.0f : 0.0f;
    const float t = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (t < 1e-4f) {
        // R = I + X + X^2 / 2 with X = [r]x; dR = E + (E X + X E) / 2, E = [e_dir]x
        float X[9] = {0, -r[2], r[1], r[2], 0, -r[0], -r[1], r[0], 0};
        float E[9] = {0, -e2, e1, e2, 0, -e0, -e1, e0, 0};
        float X2[9], EX[9], XE[9];
        mul33(X, X, X2);
        mul33(E, X, EX);
        mul33(X, E, XE);
        for (int e = 0; e < 9; ++e) {
            R[e] = ((e % 4 == 0) ? 1.0f : 0.0f) + X[e] + 0.5f * X2[e];
            dR[e] = E[e] + 0.5f * (EX[e] + XE[e]);
        }
        return;
    }
    const float it = 1.0f / t;
    const float k[3] = {r[0] * it, r[1] * it, r[2] * it};
    const float dt = (r[0] * e0 + r[1] * e1 + r[2] * e2) * it;  // d|r|
    const float dk[3] = {(e0 - k[0] * dt) * it, (e1 - k[1] * dt) * it, (e2 - k[2] * dt) * it};
    float s, c;
    sincosf(t, &s, &c);
    const float sh = sinf(0.5f * t);
    const float c1 = 2.0f * sh * sh, ds = c * dt, dc1 = s * dt;  // 1 - cos t without cancellation
    float K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    float dK[9] = {0, -dk[2], dk[1], dk[2], 0, -dk[0], -dk[1], dk[0], 0};
    float K2[9], A[9], B[9];
    mul33(K, K, K2);
    mul33(dK, K, A);
    mul33(K, dK, B);
    for (int e = 0; e < 9; ++e) {
        R[e] = ((e % 4 == 0) ? 1.0f : 0.0f) + s * K[e] + c1 * K2[e];
        dR[e] = ds * K[e] + s * dK[e] + dc1 * K2[e] + c1 * (A[e] + B[e]);
    }
}

// Camera-from-frame transforms of one instrument and their tangents along
// state direction `dir` (-1: none): T_f = T_c * T_E,f(q) (Sec. III-A.2).
__device__ void fk_tangent(const ChainDev &ch, const float *st, int dir, float (*T)[12], float (*dT)[12])
{
    float q[3], dq[3];
    for (int j = 0; j < 3; ++j) {
        const float lb = (float)ch.q_lb[j], ub = (float)ch.q_ub[j];
        if (ub == lb) {
            q[j] = lb;
            dq[j] = 0.0f;
        } else {
            const float a = 3.14159265358979f * (st[6 + j] - lb) / (ub - lb);
            float s, c;
            sincosf(a, &s, &c);
            q[j] = lb + 0.5f * (ub - lb) * (1.0f - c);       // Sec. III-A.3 inverse map
            dq[j] = (dir == 6 + j) ? 1.5707963267949f * s : 0.0f;  // d q / d qhat
        }
    }
    float R[9], dR[9];
    rotation_tangent(ch.rot_param, st, dir >= 0 && dir < 3 ? dir : -1, R, dR);
    float Tc[12] = {R[0], R[1], R[2], st[3], R[3], R[4], R[5], st[4], R[6], R[7], R[8], st[5]};
    const float dTc[12] = {dR[0], dR[1], dR[2], dir == 3 ? 1.0f : 0.0f, dR[3], dR[4], dR[5], dir == 4 ? 1.0f : 0.0f,
                           dR[6], dR[7], dR[8], dir == 5 ? 1.0f : 0.0f};
    float Tf[kMaxFrames][12], dTf[kMaxFrames][12];
    for (int f = 0; f < ch.n_frames; ++f) {
        float J[9], dJ[9];
        const float cf = (float)ch.coef[f];
        rot_axis(ch.axis[f], cf * q[ch.joint[f]], J, dJ);
        const float dang = cf * dq[ch.joint[f]];
        float L[12] = {J[0], J[1], J[2], (float)ch.offset[f][0], J[3], J[4], J[5], (float)ch.offset[f][1],
                       J[6], J[7], J[8], (float)ch.offset[f][2]};
        float dL[12] = {dJ[0] * dang, dJ[1] * dang, dJ[2] * dang, 0.0f, dJ[3] * dang, dJ[4] * dang, dJ[5] * dang,
                        0.0f, dJ[6] * dang, dJ[7] * dang, dJ[8] * dang, 0.0f};
        if (ch.axis[f] == 0)
            for (int e = 0; e < 12; ++e) dL[e] = 0.0f;
        const int p = ch.parent[f];
        if (p < 0) {
            for (int e = 0; e < 12; ++e) {
                Tf[f][e] = L[e];
                dTf[f][e] = dL[e];
            }
        } else {
            mul34(Tf[p], L, Tf[f]);
            dmul34(dTf[p], L, Tf[p], dL, dTf[f]);
        }
    }
    for (int f = 0; f < ch.n_frames; ++f) {
        mul34(Tc, Tf[f], T[f]);
        dmul34(dTc, Tf[f], Tc, dTf[f], dT[f]);
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
struct SoftArgs {
    ChainDev ch;
    int nF, nI, V, T, d, lam;
    float fx, fy, cx, cy, z_near, guard, sigma;
    int W, H, Wq, ntx, nty;
    const float4 *verts;
    const int4 *tris;
    const float *params;      // [lam * d]
    const uint32_t *mask;
    float4 *sv;               // [lam * nI * V]: u - cx, v - cy, Z, flag
    longlong2 *gv;            // [lam * nI * V]: dL/du, dL/dv in fixed point (units of 2^-32)
    float *dT;                // [lam * nI * nF * 9 * 12]
    short4 *box;              // [lam * nI * T]: window j0, i0, j1, i1 (j0 > j1: none)
    int4 *cbox;               // [lam * nchunk]: union of the windows of each chunk
    int nchunk;
    int4 *ibox;               // [lam * nI]: window of the instrument
    double *lpart;            // [lam * ntx * nty]: squared error of each tile
    float *loss;              // [lam]
    float *grad;              // [lam * d] or NULL
};

__global__ void __launch_bounds__(kSoftThreads) k_soft_project(SoftArgs a)
{
    const int c = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    __shared__ float sT[kMaxFrames][12];
    __shared__ int bx[4];
    if (tid < 4) bx[tid] = (tid < 2) ? INT_MAX : INT_MIN;
    if (tid < 32) {
        const int lane = tid, dir = lane - 1;
        float st[9];
        for (int k = 0; k < 9; ++k) st[k] = a.params[(size_t)c * a.d + 9 * b + k];
        float T[kMaxFrames][12], dT[kMaxFrames][12];
        if (lane < 10) {
            fk_tangent(a.ch, st, dir, T, dT);
            if (lane == 0)
                for (int f = 0; f < a.nF; ++f)
                    for (int e = 0; e < 12; ++e) sT[f][e] = T[f][e];
            else
                for (int f = 0; f < a.nF; ++f)
                    for (int e = 0; e < 12; ++e)
                        a.dT[((((size_t)c * a.nI + b) * a.nF + f) * 9 + dir) * 12 + e] = dT[f][e];
        }
    }
    __syncthreads();
    const float m = kSoftCutoff * a.sigma;
    int j0 = INT_MAX, i0 = INT_MAX, j1 = INT_MIN, i1 = INT_MIN;
    const size_t base = ((size_t)c * a.nI + b) * a.V;
    for (int v = tid; v < a.V; v += blockDim.x) {
        const float4 p = a.verts[v];
        const float *M = sT[(int)p.w];
        const float X = fmaf(M[0], p.x, fmaf(M[1], p.y, fmaf(M[2], p.z, M[3])));
        const float Y = fmaf(M[4], p.x, fmaf(M[5], p.y, fmaf(M[6], p.z, M[7])));
        const float Z = fmaf(M[8], p.x, fmaf(M[9], p.y, fmaf(M[10], p.z, M[11])));
        float u = 0.0f, w = 0.0f, flag = 1.0f;
        if (Z >= a.z_near) {
            u = __fdiv_rn(a.fx * X, Z);
            w = __fdiv_rn(a.fy * Y, Z);
            if (fabsf(u) <= a.guard && fabsf(w) <= a.guard) {
                flag = 0.0f;
                j0 = min(j0, (int)ceilf(u + a.cx - m));
                j1 = max(j1, (int)floorf(u + a.cx + m));
                i0 = min(i0, (int)ceilf(w + a.cy - m));
                i1 = max(i1, (int)floorf(w + a.cy + m));
            }
        }
        a.sv[base + v] = make_float4(u, w, Z, flag);
        a.gv[base + v] = make_longlong2(0, 0);
    }
    atomicMin(&bx[0], j0);
    atomicMin(&bx[1], i0);
    atomicMax(&bx[2], j1);
    atomicMax(&bx[3], i1);
    __syncthreads();
    if (tid == 0)
        a.ibox[(size_t)c * a.nI + b] = make_int4(max(bx[0], 0), max(bx[1], 0), min(bx[2], a.W - 1), min(bx[3], a.H - 1));
}

// Window of influence of every triangle (none for a flagged vertex or zero
// area), and the union of the windows of each chunk of kChunk triangles (one
// block per chunk), so that a tile skips whole chunks that cannot reach it.
__global__ void __launch_bounds__(kChunk) k_soft_tribox(SoftArgs a)
{
    const int c = blockIdx.y;
    const int NT = a.nI * a.T;
    const int t = blockIdx.x * kChunk + threadIdx.x;
    __shared__ int cb[4];
    if (threadIdx.x < 4) cb[threadIdx.x] = (threadIdx.x < 2) ? INT_MAX : INT_MIN;
    __syncthreads();
    short4 o = make_short4(1, 1, 0, 0);
    if (t < NT) {
        const int b = t >= a.T;
        const int4 tri = a.tris[t - b * a.T];
        const float4 *sv = a.sv + ((size_t)c * a.nI + b) * a.V;
        const float4 p0 = sv[tri.x], p1 = sv[tri.y], p2 = sv[tri.z];
        if (p0.w == 0.0f && p1.w == 0.0f && p2.w == 0.0f) {
            const float A = (p1.x - p0.x) * (p2.y - p0.y) - (p1.y - p0.y) * (p2.x - p0.x);
            if (A != 0.0f) {
                const float m = kSoftCutoff * a.sigma;
                const int j0 = max(0, (int)ceilf(fminf(p0.x, fminf(p1.x, p2.x)) + a.cx - m));
                const int j1 = min(a.W - 1, (int)floorf(fmaxf(p0.x, fmaxf(p1.x, p2.x)) + a.cx + m));
                const int i0 = max(0, (int)ceilf(fminf(p0.y, fminf(p1.y, p2.y)) + a.cy - m));
                const int i1 = min(a.H - 1, (int)floorf(fmaxf(p0.y, fmaxf(p1.y, p2.y)) + a.cy + m));
                if (j0 <= j1 && i0 <= i1) {
                    o = make_short4((short)j0, (short)i0, (short)j1, (short)i1);
                    atomicMin(&cb[0], j0);
                    atomicMin(&cb[1], i0);
                    atomicMax(&cb[2], j1);
                    atomicMax(&cb[3], i1);
                }
            }
        }
        a.box[(size_t)c * NT + t] = o;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.cbox[(size_t)c * a.nchunk + blockIdx.x] = make_int4(cb[0], cb[1], cb[2], cb[3]);
}

// Staged triangle: positively oriented image-space vertices, edge data, window.
struct SoftTriSmem {
    float x[3][kChunk], y[3][kChunk];
    float ex[3][kChunk], ey[3][kChunk], il[3][kChunk], il2[3][kChunk];
    short4 win[kChunk];
    int vid[3][kChunk];     // global vertex slots (into sv / gv)
    int list[kChunk];
    int wc[kChunk / 32];    // staged triangles per warp (the compaction's prefix)
    int n;
};

// Signed distance of (px, py) to staged triangle n (FP32), with the feature
// that realises it: kind 0 = edge line (inside) or segment interior
// (outside), 1 = segment start vertex, 2 = segment end vertex; k = edge.
__device__ __forceinline__ float soft_distance(const SoftTriSmem &S, int n, float px, float py, int &kind, int &kf)
{
    bool inside = true;
    float hmin = INFINITY, dmin = INFINITY;
    int kin = 0, kout = 0, kindout = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float x0 = S.x[k][n], y0 = S.y[k][n], dx = S.ex[k][n], dy = S.ey[k][n];
        const float rx = px - x0, ry = py - y0;
        const float E = fmaf(dx, ry, -dy * rx);
        const float h = E * S.il[k][n];
        if (E < 0.0f) inside = false;
        if (h < hmin) {
            hmin = h;
            kin = k;
        }
        const float s = fmaf(rx, dx, ry * dy) * S.il2[k][n];
        float dist;
        int kd;
        if (s <= 0.0f) {
            dist = sqrtf(fmaf(rx, rx, ry * ry));
            kd = 1;
        } else if (s >= 1.0f) {
            const float qx = px - (x0 + dx), qy = py - (y0 + dy);
            dist = sqrtf(fmaf(qx, qx, qy * qy));
            kd = 2;
        } else {
            dist = fabsf(h);
            kd = 0;
        }
        if (dist < dmin) {
            dmin = dist;
            kout = k;
            kindout = kd;
        }
    }
    if (inside) {
        kind = 0;
        kf = kin;
        return hmin;
    }
    kind = kindout;
    kf = kout;
    return -dmin;
}

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x))); }
__device__ __forceinline__ float sigmoidf_(float x)
{
    const float e = __expf(-fabsf(x));
    return x >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

// Stage the triangles of chunk [t0, t0 + kChunk) whose window meets the tile,
// in triangle order (a fixed order, so every sum over the staged triangles is
// the same from run to run).
__device__ void stage_chunk(const SoftArgs &a, int c, int t0, int tx0, int ty0, SoftTriSmem &S)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    const int NT = a.nI * a.T;
    const int t = t0 + tid;
    bool hit = false;
    short4 w = make_short4(1, 1, 0, 0);
    if (t < NT) {
        w = a.box[(size_t)c * NT + t];
        hit = w.x <= w.z && w.x <= tx0 + kTile - 1 && w.z >= tx0 && w.y <= ty0 + kTile - 1 && w.w >= ty0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if ((tid & 31) == 0) S.wc[warp] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int q = 0; q < warp; ++q) base += S.wc[q];
    if (tid == 0) {
        int n = 0;
        for (int q = 0; q < kChunk / 32; ++q) n += S.wc[q];
        S.n = n;
    }
    if (hit) {
        const int slot = base + __popc(bal & ((1u << (tid & 31)) - 1u));
        const int b = t >= a.T;
        const int4 tri = a.tris[t - b * a.T];
        const size_t vb = ((size_t)c * a.nI + b) * a.V;
        const float4 p0 = a.sv[vb + tri.x], p1 = a.sv[vb + tri.y], p2 = a.sv[vb + tri.z];
        const float A = (p1.x - p0.x) * (p2.y - p0.y) - (p1.y - p0.y) * (p2.x - p0.x);
        float4 q[3] = {p0, A > 0.0f ? p1 : p2, A > 0.0f ? p2 : p1};
        int id[3] = {tri.x, A > 0.0f ? tri.y : tri.z, A > 0.0f ? tri.z : tri.y};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            S.x[k][slot] = q[k].x + a.cx;
            S.y[k][slot] = q[k].y + a.cy;
            S.vid[k][slot] = (int)(vb + id[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int k1 = k == 2 ? 0 : k + 1;
            const float dx = q[k1].x - q[k].x, dy = q[k1].y - q[k].y;
            const float L2 = fmaf(dx, dx, dy * dy);
            S.ex[k][slot] = dx;
            S.ey[k][slot] = dy;
            S.il2[k][slot] = 1.0f / L2;
            S.il[k][slot] = rsqrtf(L2);
        }
        S.win[slot] = w;
    }
    __syncthreads();
}

// Does chunk k of candidate c have a window reaching the tile?
__device__ __forceinline__ bool chunk_reaches(const SoftArgs &a, int c, int k, int tx0, int ty0)
{
    const int4 b = a.cbox[(size_t)c * a.nchunk + k];
    return b.x <= b.z && b.x <= tx0 + kTile - 1 && b.z >= tx0 && b.y <= ty0 + kTile - 1 && b.w >= ty0;
}

__global__ void __launch_bounds__(kSoftThreads) k_soft_tile(SoftArgs a)
{
    const int c = blockIdx.y;
    const int tile = blockIdx.x;
    const int tx0 = (tile % a.ntx) * kTile, ty0 = (tile / a.ntx) * kTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ SoftTriSmem S;
    __shared__ float wpx[kTile * kTile];
    __shared__ float red[8];
    // this thread's pixel in the forward pass
    const int j = tx0 + (tid & (kTile - 1)), i = ty0 + tid / kTile;
    const float px = (float)j, py = (float)i, inv_s = 1.0f / a.sigma, cut = -kSoftCutoff * a.sigma;
    float acc = 0.0f;
    // is the tile within reach of any instrument?
    bool near = false;
    for (int b = 0; b < a.nI; ++b) {
        const int4 ib = a.ibox[(size_t)c * a.nI + b];
        near |= ib.x <= ib.z && ib.x <= tx0 + kTile - 1 && ib.z >= tx0 && ib.y <= ty0 + kTile - 1 && ib.w >= ty0;
    }
    if (near) {
        for (int k = 0; k < a.nchunk; ++k) {
            if (!chunk_reaches(a, c, k, tx0, ty0)) continue;  // the same decision in every thread
            stage_chunk(a, c, k * kChunk, tx0, ty0, S);
            const int n = S.n;
            for (int e = 0; e < n; ++e) {
                const short4 w = S.win[e];
                if (j < w.x || j > w.z || i < w.y || i > w.w) continue;
                int kind, kf;
                const float d = soft_distance(S, e, px, py, kind, kf);
                if (d >= cut) acc += softplusf(d * inv_s);
            }
            __syncthreads();
        }
    }
    // squared error of the tile's pixels; per-pixel factor of the backward
    float l = 0.0f, wp = 0.0f;
    if (i < a.H && j < a.W) {
        const float Sv = 1.0f - __expf(-acc);
        const float Mv = (float)((a.mask[(size_t)i * a.Wq + (j >> 5)] >> (j & 31)) & 1u);
        const float e = Sv - Mv;
        l = e * e;
        wp = 2.0f * e * (1.0f - Sv) * inv_s;
    }
    wpx[tid] = wp;
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) red[warp] = l;
    __syncthreads();
    if (tid == 0) {  // the tile's share, summed over the tiles in a fixed order by k_soft_reduce
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += (double)red[w];
        a.lpart[(size_t)c * a.ntx * a.nty + tile] = sum;
    }
    if (!a.grad || !near) return;
    // pass 2: the same pairs again, one warp per staged triangle, lanes over
    // two rows of 16 pixels at a time
    const int cj = tx0 + (lane & (kTile - 1)), rsub = lane / kTile;
    const float cpx = (float)cj;
    for (int k = 0; k < a.nchunk; ++k) {
        if (!chunk_reaches(a, c, k, tx0, ty0)) continue;
        stage_chunk(a, c, k * kChunk, tx0, ty0, S);
        const int n = S.n;
        for (int e = warp; e < n; e += 8) {
            const short4 w = S.win[e];
            float g[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const bool colin = cj >= w.x && cj <= w.z && cj < a.W;
            const int ia = max((int)w.y, ty0), ib = min((int)w.w, min(ty0 + kTile - 1, a.H - 1));
            for (int i2 = ia + rsub; i2 <= ib; i2 += 2) {
                if (!colin) break;
                int kind, kf;
                const float cpy = (float)i2;
                const float d = soft_distance(S, e, cpx, cpy, kind, kf);
                if (d < cut) continue;
                const float gd = wpx[(i2 - ty0) * kTile + (cj - tx0)] * sigmoidf_(d * inv_s);
                const int k1 = kf == 2 ? 0 : kf + 1;
                const float x0 = S.x[kf][e], y0 = S.y[kf][e], dx = S.ex[kf][e], dy = S.ey[kf][e];
                if (kind == 0) {
                    // d = E / L (inside, or outside at the segment interior: d = -|E|/L = E/L there)
                    const float E = fmaf(dx, cpy - y0, -dy * (cpx - x0));
                    const float il = S.il[kf][e], il2 = S.il2[kf][e];
                    const float h = E * il;
                    float sg = 1.0f;
                    if (d < 0.0f && E > 0.0f) sg = -1.0f;  // outside on the inner side of the line
                    const float x1 = x0 + dx, y1 = y0 + dy;
                    // d(E/L) = dE / L - (E / L^2) dL, dL = (-dx, -dy, dx, dy) / L
                    g[2 * kf] += gd * sg * ((y1 - cpy) * il + h * dx * il2);
                    g[2 * kf + 1] += gd * sg * ((cpx - x1) * il + h * dy * il2);
                    g[2 * k1] += gd * sg * ((cpy - y0) * il - h * dx * il2);
                    g[2 * k1 + 1] += gd * sg * (-(cpx - x0) * il - h * dy * il2);
                } else {
                    // d = -|p - v|: dd/dv = (p - v) / |p - v|
                    const int kv = kind == 1 ? kf : k1;
                    const float rx = cpx - S.x[kv][e], ry = cpy - S.y[kv][e];
                    const float rl = rsqrtf(fmaxf(fmaf(rx, rx, ry * ry), 1e-30f));
                    g[2 * kv] += gd * rx * rl;
                    g[2 * kv + 1] += gd * ry * rl;
                }
            }
#pragma unroll
            for (int q = 0; q < 6; ++q)
                for (int o = 16; o; o >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], o);
            if (lane < 3) {  // fixed point: the sums do not depend on the order of the additions
                unsigned long long *gp = reinterpret_cast<unsigned long long *>(a.gv + S.vid[lane][e]);
                atomicAdd(gp, (unsigned long long)to_fixed(g[2 * lane], kGvScale));
                atomicAdd(gp + 1, (unsigned long long)to_fixed(g[2 * lane + 1], kGvScale));
            }
        }
        __syncthreads();
    }
}

// Per (candidate, instrument): dL/dX of every vertex, G_f = sum over the
// frame's vertices of dL/dX [v; 1]^T, then dL/dtheta_k = sum_f <G_f, dT_f/dtheta_k>.
// Block (c, 0) also sums the candidate's tile losses in a fixed order.  Every
// sum is order-independent (fixed order, or exact fixed-point integers), so
// a call's results do not vary from run to run.
__global__ void __launch_bounds__(kSoftThreads) k_soft_reduce(SoftArgs a)
{
    const int c = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    __shared__ unsigned long long G[kMaxFrames * 12];  // fixed point, units of 2^-24
    __shared__ double red[kSoftThreads];
    if (b == 0) {
        const int nt = a.ntx * a.nty;
        double acc = 0.0;
        for (int t = tid; t < nt; t += blockDim.x) acc += a.lpart[(size_t)c * nt + t];
        red[tid] = acc;
        __syncthreads();
        for (int o = kSoftThreads / 2; o; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) a.loss[c] = (float)red[0];
    }
    if (!a.grad) return;
    for (int e = tid; e < a.nF * 12; e += blockDim.x) G[e] = 0ull;
    __syncthreads();
    const size_t base = ((size_t)c * a.nI + b) * a.V;
    // each thread sums its vertices' terms in registers while their frame stays
    // the same (a link's vertices are contiguous), then adds them to G: the
    // integer sums are exact, so grouping them changes nothing
    long long acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0;
    int fcur = -1;
    auto flush = [&]() {
        if (fcur < 0) return;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            if (acc[k]) atomicAdd(G + fcur * 12 + k, (unsigned long long)acc[k]);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = 0;
    };
    for (int v = tid; v < a.V; v += blockDim.x) {
        const float4 s = a.sv[base + v];
        const longlong2 q = a.gv[base + v];
        if (s.w != 0.0f || (q.x == 0 && q.y == 0)) continue;
        const float gx = (float)((double)q.x * (1.0 / kGvScale)), gy = (float)((double)q.y * (1.0 / kGvScale));
        const float iz = 1.0f / s.z;
        const float gX = gx * a.fx * iz, gY = gy * a.fy * iz, gZ = -(gx * s.x + gy * s.y) * iz;
        const float4 p = a.verts[v];
        const int f = (int)p.w;
        if (f != fcur) {
            flush();
            fcur = f;
        }
        const float vh[4] = {p.x, p.y, p.z, 1.0f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k] += to_fixed(gX * vh[k], kGScale);
            acc[4 + k] += to_fixed(gY * vh[k], kGScale);
            acc[8 + k] += to_fixed(gZ * vh[k], kGScale);
        }
    }
    flush();
    __syncthreads();
    if (tid < 9) {
        float acc = 0.0f;
        for (int f = 0; f < a.nF; ++f) {
            const float *dT = a.dT + ((((size_t)c * a.nI + b) * a.nF + f) * 9 + tid) * 12;
            for (int e = 0; e < 12; ++e)
                acc = fmaf((float)((double)(long long)G[f * 12 + e] * (1.0 / kGScale)), dT[e], acc);
        }
        a.grad[(size_t)c * a.d + 9 * b + tid] = acc;
    }
}


// Adam on the refined candidates, in the optimiser's normalised units
// (x = params / scales): m, v, bias correction (Kingma & Ba, 2015).
__global__ void k_adam(float *P, const float *g, float *m, float *v, const CmaConst *k, int n, int d, float lr,
                       float b1, float b2, float eps, int step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * d) return;
    const float sc = (float)k->scales[i % d];
    const float gn = g[i] * sc;
    const float mi = b1 * m[i] + (1.0f - b1) * gn;
    const float vi = b2 * v[i] + (1.0f - b2) * gn * gn;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)step)), vh = vi / (1.0f - powf(b2, (float)step));
    P[i] -= lr * sc * mh / (sqrtf(vh) + eps);
}

// The k best candidates of the last generation (by loss, then index) into P;
// Adam moments cleared.
__global__ void k_refine_init(const float *params, const float *loss, int lam, int d, int kk, float *P, float *m,
                              float *v, int *order)
{
    __shared__ int sel[32];
    if (threadIdx.x == 0) {
        for (int r = 0; r < kk; ++r) {
            int best = -1;
            for (int c = 0; c < lam; ++c) {
                bool taken = false;
                for (int q = 0; q < r; ++q) taken |= sel[q] == c;
                if (taken) continue;
                if (best < 0 || loss[c] < loss[best]) best = c;  // ties keep the lower index
            }
            sel[r] = best;
            order[r] = best;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kk * d; e += blockDim.x) {
        P[e] = params[(size_t)sel[e / d] * d + e % d];
        m[e] = 0.0f;
        v[e] = 0.0f;
    }
}

// The refined candidate with the lowest fitness loss (ties: lower index)
// replaces the frame's estimate when it beats the frame's best.
__global__ void k_refine_pick(const float *P, const float *lhard, int kk, int d, CmaState *st, float *pose_out,
                              int *picked)
{
    __shared__ int best;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int r = 1; r < kk; ++r)
            if (lhard[r] < lhard[b]) b = r;
        best = (lhard[b] < st->best_loss) ? b : -1;
        *picked = best;
        if (best >= 0) st->best_loss = lhard[b];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        if (best >= 0) {
            const float x = P[(size_t)best * d + i];
            st->best_x[i] = x;
            st->est[i] = (double)x;
        }
        if (pose_out) pose_out[i] = (float)st->est[i];
    }
}

}  // namespace trk

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using namespace trk;

namespace {

struct SoftScratch {
    int cap = 0;
    float4 *sv = nullptr;
    longlong2 *gv = nullptr;
    float *dT = nullptr;
    short4 *box = nullptr;
    int4 *ibox = nullptr;
    int4 *cbox = nullptr;
    double *lpart = nullptr;
    int lpart_cap = 0;
};

struct RefineBuf {
    int cap = 0;
    float *P = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *ls = nullptr, *lh = nullptr;
    int *order = nullptr, *picked = nullptr;
};

trk_status soft_fail(trk_status st, const char *why)
{
    set_last_error(why);
    return st;
}

trk_status soft_scratch(trk_tracker *t, int lam, SoftScratch **out)
{
    SoftScratch *s = static_cast<SoftScratch *>(t->soft);
    if (s && s->cap >= lam) {
        *out = s;
        return TRK_OK;
    }
    soft_free(t);
    s = new SoftScratch();
    const int nI = t->ch.n_inst;
    const size_t nv = (size_t)lam * nI * t->V;
    cudaError_t e;
    if ((e = cudaMalloc(&s->sv, sizeof(float4) * nv)) != cudaSuccess ||
        (e = cudaMalloc(&s->gv, sizeof(longlong2) * nv)) != cudaSuccess ||
        (e = cudaMalloc(&s->dT, sizeof(float) * (size_t)lam * nI * t->ch.n_frames * 9 * 12)) != cudaSuccess ||
        (e = cudaMalloc(&s->box, sizeof(short4) * (size_t)lam * nI * t->T)) != cudaSuccess ||
        (e = cudaMalloc(&s->ibox, sizeof(int4) * (size_t)lam * nI)) != cudaSuccess ||
        (e = cudaMalloc(&s->cbox, sizeof(int4) * (size_t)lam * ((nI * t->T + kChunk - 1) / kChunk))) != cudaSuccess ||
        (e = cudaMalloc(&s->lpart, sizeof(double) * lam * (size_t)((t->cam.W + kTile - 1) / kTile) *
                                       ((t->cam.H + kTile - 1) / kTile))) != cudaSuccess) {
        t->soft = s;
        soft_free(t);
        return soft_fail(e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA, cudaGetErrorString(e));
    }
    s->cap = lam;
    s->lpart_cap = lam;
    t->soft = s;
    *out = s;
    return TRK_OK;
}

trk_status soft_launch(trk_tracker *t, const float *params, int lam, const uint32_t *mask, float sigma, float *loss,
                       float *grad, cudaStream_t st)
{
    if (lam == 0) return TRK_OK;
    SoftScratch *s = nullptr;
    trk_status r = soft_scratch(t, lam, &s);
    if (r != TRK_OK) return r;
    SoftArgs a{};
    a.ch = t->ch;
    a.nF = t->ch.n_frames;
    a.nI = t->ch.n_inst;
    a.V = t->V;
    a.T = t->T;
    a.d = t->d;
    a.lam = lam;
    a.fx = (float)t->cam.fx;
    a.fy = (float)t->cam.fy;
    a.cx = (float)(t->cam.cx256 / 256.0);
    a.cy = (float)(t->cam.cy256 / 256.0);
    a.z_near = (float)t->cam.z_near;
    a.guard = (float)t->cam.guard;
    a.sigma = sigma;
    a.W = t->cam.W;
    a.H = t->cam.H;
    a.Wq = t->cam.Wq;
    a.ntx = (a.W + kTile - 1) / kTile;
    a.nty = (a.H + kTile - 1) / kTile;
    a.verts = t->verts;
    a.tris = t->tris;
    a.params = params;
    a.mask = mask;
    a.sv = s->sv;
    a.gv = s->gv;
    a.dT = s->dT;
    a.box = s->box;
    a.ibox = s->ibox;
    a.lpart = s->lpart;
    a.cbox = s->cbox;
    a.nchunk = (a.nI * a.T + kChunk - 1) / kChunk;
    a.loss = loss;
    a.grad = grad;
    k_soft_project<<<dim3(lam, a.nI), kSoftThreads, 0, st>>>(a);
    k_soft_tribox<<<dim3(a.nchunk, lam), kChunk, 0, st>>>(a);
    k_soft_tile<<<dim3(a.ntx * a.nty, lam), kSoftThreads, 0, st>>>(a);
    k_soft_reduce<<<dim3(lam, a.nI), kSoftThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TRK_OK : soft_fail(TRK_ECUDA, cudaGetErrorString(e));
}

}  // namespace

void trk::soft_free(trk_tracker *t)
{
    SoftScratch *s = static_cast<SoftScratch *>(t->soft);
    if (!s) return;
    cudaFree(s->sv);
    cudaFree(s->gv);
    cudaFree(s->dT);
    cudaFree(s->box);
    cudaFree(s->ibox);
    cudaFree(s->cbox);
    cudaFree(s->lpart);
    delete s;
    t->soft = nullptr;
}

void trk::refine_free(trk_cmaes *es)
{
    RefineBuf *r = static_cast<RefineBuf *>(es->refine);
    if (!r) return;
    cudaFree(r->P);
    cudaFree(r->g);
    cudaFree(r->m);
    cudaFree(r->v);
    cudaFree(r->ls);
    cudaFree(r->lh);
    cudaFree(r->order);
    cudaFree(r->picked);
    delete r;
    es->refine = nullptr;
}

extern "C" {

trk_status soft_eval(trk_tracker *t, const float *params_dev, int32_t lam, const uint32_t *mask_packed_dev,
                     float sigma, float *loss_dev, float *grad_dev, void *stream)
{
    if (!t) return soft_fail(TRK_EINVAL, "NULL tracker");
    if (lam < 0 || lam > TRK_MAX_LAMBDA) return soft_fail(TRK_EINVAL, "lam out of range");
    if (lam == 0) return TRK_OK;
    if (!params_dev || !mask_packed_dev || !loss_dev) return soft_fail(TRK_EINVAL, "NULL device pointer");
    if (!(sigma >= 0.05f && sigma <= 64.0f)) return soft_fail(TRK_EINVAL, "sigma must be in [0.05, 64] px");
    if (t->cam.W > 32767 || t->cam.H > 32767) return soft_fail(TRK_EINVAL, "image too large");
    return soft_launch(t, params_dev, lam, mask_packed_dev, sigma, loss_dev, grad_dev,
                       reinterpret_cast<cudaStream_t>(stream));
}

trk_status soft_refine(trk_cmaes *es, const uint32_t *mask_packed_dev, int32_t top_k, int32_t steps, float lr,
                       float sigma, float *pose_out_dev, int32_t *picked_host, void *stream)
{
    if (!es || !mask_packed_dev) return soft_fail(TRK_EINVAL, "NULL argument");
    if (top_k < 1 || top_k > 32 || top_k > es->lam) return soft_fail(TRK_EINVAL, "top_k must be 1..min(32, lam)");
    if (steps < 0 || steps > 1000) return soft_fail(TRK_EINVAL, "steps out of range");
    if (!(lr > 0.0f && lr < 10.0f)) return soft_fail(TRK_EINVAL, "lr out of range");
    if (!(sigma >= 0.05f && sigma <= 64.0f)) return soft_fail(TRK_EINVAL, "sigma must be in [0.05, 64] px");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    trk_tracker *t = es->t;
    RefineBuf *r = static_cast<RefineBuf *>(es->refine);
    if (!r) {
        r = new RefineBuf();
        const size_t n = (size_t)32 * es->d;
        cudaError_t e;
        if ((e = cudaMalloc(&r->P, sizeof(float) * n)) != cudaSuccess ||
            (e = cudaMalloc(&r->g, sizeof(float) * n)) != cudaSuccess ||
            (e = cudaMalloc(&r->m, sizeof(float) * n)) != cudaSuccess ||
            (e = cudaMalloc(&r->v, sizeof(float) * n)) != cudaSuccess ||
            (e = cudaMalloc(&r->ls, sizeof(float) * 32)) != cudaSuccess ||
            (e = cudaMalloc(&r->lh, sizeof(float) * 32)) != cudaSuccess ||
            (e = cudaMalloc(&r->order, sizeof(int) * 32)) != cudaSuccess ||
            (e = cudaMalloc(&r->picked, sizeof(int))) != cudaSuccess) {
            es->refine = r;
            refine_free(es);
            return soft_fail(e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA, cudaGetErrorString(e));
        }
        r->cap = 32;
        es->refine = r;
    }
    const int d = es->d;
    k_refine_init<<<1, 128, 0, s>>>(es->params, es->loss, es->lam, d, top_k, r->P, r->m, r->v, r->order);
    for (int step = 1; step <= steps; ++step) {
        trk_status st = soft_launch(t, r->P, top_k, mask_packed_dev, sigma, r->ls, r->g, s);
        if (st != TRK_OK) return st;
        k_adam<<<(top_k * d + 127) / 128, 128, 0, s>>>(r->P, r->g, r->m, r->v, es->k, top_k, d, lr, 0.9f, 0.999f,
                                                       1e-8f, step);
    }
    // fitness (binary silhouette, the tracker's loss) of the refined candidates
    EvalArgs a{};
    a.ch = t->ch;
    a.cam = t->cam;
    apply_mesh(a, t);
    a.params = r->P;
    a.d = d;
    a.lam = top_k;
    a.mask = mask_packed_dev;
    a.snap = t->snap;
    a.loss = r->lh;
    a.loss_kind = t->cfg.loss_kind;
    a.lambda_app = t->cfg.lambda_app;
    a.cull = t->cfg.cull_backfaces;
    apply_keypoints(a, t);
    cudaError_t e = launch_eval(a, t->lc, s);
    if (e != cudaSuccess) return soft_fail(TRK_ECUDA, cudaGetErrorString(e));
    k_refine_pick<<<1, 32, 0, s>>>(r->P, r->lh, top_k, d, es->st, pose_out_dev, r->picked);
    if ((e = cudaGetLastError()) != cudaSuccess) return soft_fail(TRK_ECUDA, cudaGetErrorString(e));
    if (picked_host) {
        if ((e = cudaMemcpyAsync(picked_host, r->picked, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return soft_fail(TRK_ECUDA, cudaGetErrorString(e));
    }
    return TRK_OK;
}

}  // extern "C"
