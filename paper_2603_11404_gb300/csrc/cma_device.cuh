// Device-side CMA-ES building blocks (arXiv 2603.11404, Sec. III-A.1,
// Eq. cmaes_update; block-diagonal form of Sec. III-B), shared by the
// stand-alone CMA-ES kernels and the fused per-generation fitness kernel.
//
// Precision plan (GB300's FP64 pipe is narrow and slow: a dependent FP64 FMA
// costs ~64 cycles, division and square root ~700): the covariance, paths and
// step size are FP64; sampling draws FP32 normals; the eigendecomposition runs
// a warm-started FP32 Jacobi pass for the bulk of the rotation, then makes the
// basis orthogonal in FP64 (Newton-Schulz), and C^(1/2), C^(-1/2) come from
// the nearly diagonal V^T C V by two Newton steps for the matrix square root
// (Sylvester equations solved entrywise), accurate to FP64 rounding without
// FP64 Jacobi sweeps, divisions or square roots in loops.
#pragma once

#include <math.h>

#include "df.cuh"
#include "internal.cuh"

namespace trk {

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Four standard normals from counter block `blk` of (seed, stream, generation):
// 24-bit uniforms u = ((r >> 8) + 1/2) 2^-24 and the Box-Muller transform in
// FP32 (the oracle evaluates the same formula in FP64).
__device__ __forceinline__ void normals4(unsigned long long seed, unsigned stream, unsigned gen, unsigned blk,
                                         float z[4])
{
    uint32_t c[4] = {blk, gen, stream, 0u};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    const float s24 = 5.9604644775390625e-8f;  // 2^-24
    float u0 = ((float)(c[0] >> 8) + 0.5f) * s24;
    float u1 = ((float)(c[1] >> 8) + 0.5f) * s24;
    float u2 = ((float)(c[2] >> 8) + 0.5f) * s24;
    float u3 = ((float)(c[3] >> 8) + 0.5f) * s24;
    float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0, s1, c1;
    sincospif(2.0f * u1, &s0, &c0);
    sincospif(2.0f * u3, &s1, &c1);
    z[0] = r0 * c0;
    z[1] = r0 * s0;
    z[2] = r1 * c1;
    z[3] = r1 * s1;
}

// Forward cosine map of Sec. III-A.3 (joint reading q -> unconstrained q-hat).
__device__ __forceinline__ double qhat_from_q(double q, double lb, double ub)
{
    if (ub == lb) return lb;
    double a = 1.0 - 2.0 * (q - lb) / (ub - lb);
    a = fmin(1.0, fmax(-1.0, a));
    return lb + (ub - lb) / M_PI * acos(a);
}

// Sample candidate kk with one warp: x = m + sigma C^(1/2) z in double-float
// arithmetic (FP32 pipes) from FP32 normals or the caller's normals z_in,
// params = x * scales rounded to FP32; y = C^(1/2) z is kept in FP64 for the
// update.  Outputs that are NULL are skipped; zs is d float2 of warp scratch.
__device__ __forceinline__ void cma_sample_warp(const CmaConst &k, const CmaState *st, int kk, const double *z_in,
                                                double *y_out, double *z_out, float *params_out, float *params_smem,
                                                float2 *zs, int lane)
{
    const int d = k.d;
    if (lane < d) {
        float2 z;
        if (z_in) {
            z = split_df(z_in[(size_t)kk * d + lane]);
        } else {
            int n = kk * d + lane;
            float zb[4];
            normals4(k.seed, k.stream_id, (unsigned)st->gen_total, (unsigned)(n >> 2), zb);
            z = make_float2(zb[n & 3], 0.0f);
        }
        zs[lane] = z;
    }
    __syncwarp();
    if (lane < d) {
        float2 row[kMaxD];  // issue all loads of the C^(1/2) row before the chain
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) row[j] = (j < d) ? st->C_half_df[lane * d + j] : make_float2(0.f, 0.f);
        dfl acc = df_from(0.0f);
#pragma unroll
        for (int j = 0; j < kMaxD; ++j)
            if (j < d) acc = df_fma(dfl{row[j].x, row[j].y}, dfl{zs[j].x, zs[j].y}, acc);
        float2 mdf = st->m_df[lane], sdf = st->sigma_df, cdf = k.scales_df[lane];
        dfl x = df_fma(dfl{sdf.x, sdf.y}, acc, dfl{mdf.x, mdf.y});
        float p = df_mul(x, dfl{cdf.x, cdf.y}).hi;
        if (params_smem) params_smem[lane] = p;
        if (y_out) y_out[(size_t)kk * d + lane] = (double)acc.hi + (double)acc.lo;
        if (z_out) z_out[(size_t)kk * d + lane] = (double)zs[lane].x + (double)zs[lane].y;
        if (params_out) params_out[(size_t)kk * d + lane] = p;
    }
    __syncwarp();
}

// Shared memory of one update; the selected steps are staged in shared memory
// when mu * d <= kYselCap (populations up to lam = 128 at d = 18, 256 at d = 9).
constexpr int kYselCap = 64 * kMaxD;
struct TellSmem {
    float sl[TRK_MAX_LAMBDA];
    int order[TRK_MAX_LAMBDA];
    double yw[kMaxD], pc[kMaxD], sq[kMaxD], isq[kMaxD];
    double part[8][kMaxD];
    double C[kMaxD * kMaxD], A[kMaxD * kMaxD], A2[kMaxD * kMaxD], V[kMaxD * kMaxD], V2[kMaxD * kMaxD];
    double B[kMaxD * kMaxD], ysel[kYselCap], w[TRK_MAX_LAMBDA / 2];
    float Af[kMaxD * kMaxD], Vf[kMaxD * kMaxD], Vf2[kMaxD * kMaxD];
    double n2, hs;
};

// C (d x d, FP64, row-major) -> out = X^T C X for square X, FP64.
// 1 / a for a > 0 in FP64 without a division: the FP32 reciprocal as a seed,
// then two Newton-Raphson steps r <- r + r (1 - a r), each doubling the
// correct bits (24 -> 48 -> 96, so the result is correctly rounded or 1 ulp off).
__device__ __forceinline__ double rcp64(double a)
{
    double r = (double)__frcp_rn((float)a);
    r = __fma_rn(r, __fma_rn(-a, r, 1.0), r);
    r = __fma_rn(r, __fma_rn(-a, r, 1.0), r);
    return r;
}

__device__ __forceinline__ void sandwich64(int d, const double *X, const double *Cm, double *tmp, double *out, int tid,
                                           int nt)
{
    for (int e = tid; e < d * d; e += nt) {
        int i = e / d, j = e - i * d;
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = __fma_rn(Cm[i * d + q], X[q * d + j], acc);
        tmp[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < d * d; e += nt) {
        int i = e / d, j = e - i * d;
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = __fma_rn(X[q * d + i], tmp[q * d + j], acc);
        out[e] = acc;
    }
    __syncthreads();
}

// One-sided Jacobi, columns in shared memory (any d): Xc, Jc column-major
// d x d; called by one warp.
template <int D>  // D > 0: the dimension as a compile-time constant (cheap index arithmetic)
static __device__ __noinline__ void onesided_jacobi_smem(float *Xc, float *Jc, int dyn_d, int lane, CmaState *st)
{
    const int d = D > 0 ? D : dyn_d, n2 = d + (d & 1);
    float amax = 0.0f;  // largest squared column norm, for the absolute floor
    if (lane < d)
        for (int q = 0; q < d; ++q) amax = fmaxf(amax, Xc[lane * d + q] * Xc[lane * d + q]);
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    int sweeps = 0;
    for (; sweeps < 12; ++sweeps) {
        bool rotated = false;
        float rho = 0.0f;  // largest |u . w| / (|u| |w|) rotated in this sweep
        for (int r = 0; r < n2 - 1; ++r) {
            // circle method: position n2-1 meets r, the others pair as (r+i, r-i) mod n2-1
            int partner;
            if (lane == n2 - 1) partner = r;
            else if (lane == r) partner = n2 - 1;
            else partner = (2 * r - lane + 2 * (n2 - 1)) % (n2 - 1);
            const bool act = lane < d && partner < d;
            const int lo = min(lane, partner), hi = max(lane, partner);
            float c = 1.0f, sn = 0.0f;
            float xo[kMaxD], vo[kMaxD];
            if (act) {
                float a = 0.0f, b = 0.0f, g = 0.0f;
#pragma unroll
                for (int q = 0; q < kMaxD; ++q)
                    if (q < d) {
                        const float u = Xc[lo * d + q], w = Xc[hi * d + q];
                        a = fmaf(u, u, a);
                        b = fmaf(w, w, b);
                        g = fmaf(u, w, g);
                    }
                if (g * g > 1e-10f * a * b + 1e-22f * amax * amax) {
                    // approximate intrinsics are enough: any rotation close to the
                    // annihilating one converges, and the test above uses exact g, a, b
                    const float zeta = __fdividef(b - a, 2.0f * g), h = fmaf(zeta, zeta, 1.0f);
                    const float t = copysignf(__fdividef(1.0f, fabsf(zeta) + h * rsqrtf(h)), zeta);
                    c = rsqrtf(1.0f + t * t);
                    sn = t * c;
                    rotated = true;
                    rho = fmaxf(rho, fabsf(g) * rsqrtf(a * b));
                }
                // own column after the rotation: lo gets c u - s w, hi gets s u + c w
                const bool is_lo = lane == lo;
#pragma unroll
                for (int q = 0; q < kMaxD; ++q)
                    if (q < d) {
                        const float u = Xc[lo * d + q], w = Xc[hi * d + q];
                        const float ju = Jc[lo * d + q], jw = Jc[hi * d + q];
                        xo[q] = is_lo ? fmaf(c, u, -sn * w) : fmaf(sn, u, c * w);
                        vo[q] = is_lo ? fmaf(c, ju, -sn * jw) : fmaf(sn, ju, c * jw);
                    }
            }
            __syncwarp();
            if (act) {
#pragma unroll
                for (int q = 0; q < kMaxD; ++q)
                    if (q < d) {
                        Xc[lane * d + q] = xo[q];
                        Jc[lane * d + q] = vo[q];
                    }
            }
            __syncwarp();
        }
        // Jacobi converges quadratically: after a sweep whose rotations were
        // all below 3e-3 the columns are orthogonal to ~1e-5 without checking
        for (int o = 16; o; o >>= 1) rho = fmaxf(rho, __shfl_xor_sync(0xffffffffu, rho, o));
        if (!__any_sync(0xffffffffu, rotated) || rho < 3e-3f) {
            ++sweeps;
            break;
        }
    }
    if (lane == 0) st->jacobi_sweeps = sweeps;
    }

// The same with the columns in registers (small compile-time D): lane j holds
// column j of X and of J, and a round exchanges columns by warp shuffles.
template <int D>
__device__ __forceinline__ void onesided_jacobi_regs(float *Xc, int lane, CmaState *st)
{
    // Only the columns are rotated: once they are orthogonal, column j of
    // X = C B J is C v_j = lambda_j v_j for the eigenvector v_j = (B J)_j, so
    // the caller recovers the basis by normalising the columns and the
    // accumulated rotation J is never needed.
    constexpr int N2 = D + (D & 1);
    float x[D];
#pragma unroll
    for (int q = 0; q < D; ++q) x[q] = lane < D ? Xc[lane * D + q] : 0.0f;
    float amax = 0.0f;
#pragma unroll
    for (int q = 0; q < D; ++q) amax = fmaxf(amax, x[q] * x[q]);
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float floor2 = 1e-22f * amax * amax;
    int sweeps = 0;
    for (; sweeps < 12; ++sweeps) {
        bool rotated = false;
        float rho = 0.0f;
#pragma unroll
        for (int r = 0; r < N2 - 1; ++r) {
            int partner = lane;
            if (lane < N2) {
                if (lane == N2 - 1) partner = r;
                else if (lane == r) partner = N2 - 1;
                else partner = (2 * r - lane + 2 * (N2 - 1)) % (N2 - 1);
            }
            const bool act = lane < D && partner < D;
            const int src = act ? partner : lane;
            float px[D];
#pragma unroll
            for (int q = 0; q < D; ++q) px[q] = __shfl_sync(0xffffffffu, x[q], src);
            if (act) {
                const bool is_lo = lane < partner;
                // |u|^2, |w|^2, u . w (u = lo, w = hi), each as two interleaved chains
                float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f, g0 = 0.0f, g1 = 0.0f;
#pragma unroll
                for (int q = 0; q < D; q += 2) {
                    const float u = is_lo ? x[q] : px[q], w = is_lo ? px[q] : x[q];
                    a0 = fmaf(u, u, a0);
                    b0 = fmaf(w, w, b0);
                    g0 = fmaf(u, w, g0);
                    if (q + 1 < D) {
                        const float u1 = is_lo ? x[q + 1] : px[q + 1], w1 = is_lo ? px[q + 1] : x[q + 1];
                        a1 = fmaf(u1, u1, a1);
                        b1 = fmaf(w1, w1, b1);
                        g1 = fmaf(u1, w1, g1);
                    }
                }
                const float a = a0 + a1, b = b0 + b1, g = g0 + g1;
                if (g * g > 1e-10f * a * b + floor2) {
                    // the rotation that makes u . w = 0, by its double angle:
                    // cos 2th = |b - a| / h, sin 2th = sgn((b - a) g) 2|g| / h with
                    // h = sqrt((b - a)^2 + 4 g^2), |th| <= pi/4; then
                    // c = sqrt((1 + cos 2th) / 2), s = sin 2th / (2 c) -- two
                    // reciprocal square roots in sequence.  Approximate intrinsics
                    // are enough: any rotation close to the annihilating one
                    // converges, and the test above uses exact g, a, b
                    const float dba = b - a;
                    const float ih = rsqrtf(fmaf(dba, dba, 4.0f * g * g));
                    const float c2 = fmaf(0.5f * fabsf(dba), ih, 0.5f);  // (1 + cos 2th) / 2, in [1/2, 1]
                    const float ic = rsqrtf(c2);
                    const float c = c2 * ic;
                    const float sn = copysignf(1.0f, dba) * g * ih * ic;  // sin 2th / (2 c)
                    rotated = true;
                    rho = fmaxf(rho, fabsf(g) * rsqrtf(a * b));
                    const float cu = is_lo ? c : sn, cw = is_lo ? -sn : c;  // own = cu u + cw w
#pragma unroll
                    for (int q = 0; q < D; ++q) {
                        const float u = is_lo ? x[q] : px[q], w = is_lo ? px[q] : x[q];
                        x[q] = fmaf(cu, u, cw * w);
                    }
                }
            }
        }
        for (int o = 16; o; o >>= 1) rho = fmaxf(rho, __shfl_xor_sync(0xffffffffu, rho, o));
        if (!__any_sync(0xffffffffu, rotated) || rho < 3e-3f) {
            ++sweeps;
            break;
        }
    }
    if (lane < D)
#pragma unroll
        for (int q = 0; q < D; ++q) Xc[lane * D + q] = x[q];
    if (lane == 0) st->jacobi_sweeps = sweeps;
    __syncwarp();
}

// The whole update from the fitness of the last population (called by every
// thread of one block).  y [lam*d] are the FP64 steps of that population.
// DC is the dimension as a compile-time constant (0 = read k.d at run time):
// the index arithmetic below divides by d and by the number of Jacobi pairs,
// which is cheap only for constant divisors.
template <int DC>
__device__ __forceinline__ void cma_sqrt_phases(const CmaConst &k, CmaState *st, TellSmem &S, int tid, int nt,
                                                bool do_sigma, double sigma);

// The step-size update (cumulative step-size adaptation) and the generation
// counters, from |p_sigma|^2 in S.n2.
__device__ __forceinline__ void cma_sigma_step(const CmaConst &k, CmaState *st, double n2, double sigma)
{
    double sg = sigma * exp(k.cs_over_ds * (sqrt(n2) * k.inv_chi - 1.0));
    st->sigma = sg;
    st->sigma_df = split_df(sg);
    st->gen += 1;
    st->gen_total += 1;
}

// do_sqrt = false leaves C^(1/2), C^(-1/2) and the eigenbasis as they were
// (the caller either resets the search next or runs cma_sqrt_block first).
template <int DC>
__device__ __forceinline__ void cma_tell_impl(const CmaConst &k, CmaState *st, const double *y, const float *params,
                                              const float *loss, TellSmem &S, int tid, int nt, bool do_sqrt)
{
    const int d = DC ? DC : k.d, lam = k.lam, dd = d * d, mu = k.mu;
    for (int i = tid; i < lam; i += nt) {
        float v = loss[i];
        S.sl[i] = isnan(v) ? INFINITY : v;
    }
    for (int e = tid; e < dd; e += nt) {
        S.C[e] = st->C[e];
        S.B[e] = st->C_inv_half[e];  // S.B: the eigen fallback reloads the basis itself
    }
    for (int r = tid; r < mu; r += nt) S.w[r] = k.w[r];
    __syncthreads();
    // stable ranking by (loss, index); a candidate that is selected (rank < mu)
    // stages its step y in shared memory at its rank when the selected steps
    // fit (its loads are issued before the ranking count, which hides them)
    const bool staged = mu * d <= kYselCap;
    for (int i = tid; i < lam; i += nt) {
        double yi[kMaxD];
        if (staged)
#pragma unroll
            for (int q = 0; q < kMaxD; ++q)
                if (q < d) yi[q] = y[(size_t)i * d + q];
        float li = S.sl[i];
        int r = 0;
        for (int j = 0; j < lam; ++j) {
            float lj = S.sl[j];
            r += (lj < li) || (lj == li && j < i);
        }
        S.order[r] = i;
        if (staged && r < mu)
#pragma unroll
            for (int q = 0; q < kMaxD; ++q)
                if (q < d) S.ysel[r * d + q] = yi[q];
    }
    __syncthreads();
    if (tid >= nt - 32) {  // the frame's best so far, on the last warp (the mean's partial sums start on the first)
        const int lane = tid - (nt - 32), b = S.order[0];
        const float prev = st->best_loss;
        __syncwarp();
        if (S.sl[b] < prev) {
            for (int i = lane; i < d; i += 32) st->best_x[i] = params[(size_t)b * d + i];
            if (lane == 0) st->best_loss = S.sl[b];
        }
    }
#define YSEL(r, i) (staged ? S.ysel[(r) * d + (i)] : y[(size_t)S.order[r] * d + (i)])
    // <y>_w = sum_{r < mu} w_r y_{r:lam}: 8 deterministic partial sums per coordinate
    const int chunk = (mu + 7) / 8;
    for (int e = tid; e < 8 * d; e += nt) {
        int part = e / d, i = e - part * d;
        double acc = 0.0;
        int r1 = min(mu, (part + 1) * chunk);
        for (int r = part * chunk; r < r1; ++r) acc = __fma_rn(S.w[r], YSEL(r, i), acc);
        S.part[part][i] = acc;
    }
    __syncthreads();
    // The mean, the evolution paths and h_sigma in warp 0 (lanes = coordinates,
    // d <= 32, shuffles instead of block barriers) while the other warps form
    // the rank-mu sums: C <- decay C + c1 p_c p_c^T + c_mu sum w_r y_r y_r^T
    // (block form: zero off-diagonal blocks), as 4 deterministic partial chains
    // per upper-triangle entry in the (still unused) A, A2, V, V2 buffers
    const double sigma = st->sigma, cs = k.c_sigma, cc = k.c_c;
    const double c1 = k.c_1, cmu = k.c_mu;
    double *part4[4] = {S.A, S.A2, S.V, S.V2};
    const int nup = d * (d + 1) / 2;  // entries (i, j), j >= i
    const bool split = nt > 32;  // warp 0 takes the paths, the rest the rank-mu sums
    if (tid < 32) {
        const int lane = tid;
        const bool on = lane < d;
        double yw = 0.0;
        if (on) {  // <y>_w from the 8 partial sums, as a fixed tree
            const double a = __dadd_rn(S.part[0][lane], S.part[1][lane]), b = __dadd_rn(S.part[2][lane], S.part[3][lane]);
            const double c = __dadd_rn(S.part[4][lane], S.part[5][lane]), e = __dadd_rn(S.part[6][lane], S.part[7][lane]);
            yw = __dadd_rn(__dadd_rn(a, b), __dadd_rn(c, e));
        }
        // (C^(-1/2) <y>_w)_lane in three chains
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int j = 0; j < d; j += 3) {
            const double y0 = __shfl_sync(0xffffffffu, yw, j);
            const double y1 = __shfl_sync(0xffffffffu, yw, j + 1 < d ? j + 1 : 0);
            const double y2 = __shfl_sync(0xffffffffu, yw, j + 2 < d ? j + 2 : 0);
            if (on) {
                t0 = __fma_rn(S.B[lane * d + j], y0, t0);
                if (j + 1 < d) t1 = __fma_rn(S.B[lane * d + j + 1], y1, t1);
                if (j + 2 < d) t2 = __fma_rn(S.B[lane * d + j + 2], y2, t2);
            }
        }
        const double t = __dadd_rn(__dadd_rn(t0, t1), t2);
        double ps = 0.0;
        if (on) {
            ps = __dadd_rn(__dmul_rn(1.0 - cs, st->p_sigma[lane]), __dmul_rn(k.ps_coef, t));
            st->p_sigma[lane] = ps;
            const double mn = __dadd_rn(st->m[lane], __dmul_rn(k.c_m * sigma, yw));
            st->m[lane] = mn;
            st->m_df[lane] = split_df(mn);
        }
        double n2 = ps * ps;  // |p_sigma|^2 by a fixed butterfly
        for (int o = 16; o; o >>= 1) n2 = __dadd_rn(n2, __shfl_xor_sync(0xffffffffu, n2, o));
        // h_sigma: |p_sigma| / sqrt(1 - (1 - c_sigma)^(2(g+1))) < (1.4 + 2/(n+1)) chi_n, compared squared
        const double pw = st->cs_pow * (1.0 - cs) * (1.0 - cs);
        const double hs = (n2 < k.hs_thr2 * (1.0 - pw)) ? 1.0 : 0.0;
        if (lane == 0) {
            S.n2 = n2;
            S.hs = hs;
        }
        __syncwarp();
        if (lane == 0) st->cs_pow = pw;
        if (on) {
            const double v = __dadd_rn(__dmul_rn(1.0 - cc, st->p_c[lane]), __dmul_rn(hs * k.pc_coef, yw));
            st->p_c[lane] = v;
            S.pc[lane] = v;
        }
    }
    if (!split || tid >= 32) {
        const int rchunk = (mu + 3) / 4;
        for (int e = split ? tid - 32 : tid; e < 4 * nup; e += split ? nt - 32 : nt) {
            const int pr = e / nup;
            int u = e - pr * nup, i = 0;
            while (u >= d - i) {  // row i holds d - i entries of the upper triangle
                u -= d - i;
                ++i;
            }
            const int j = i + u, ij = i * d + j;
            double rmu = 0.0;
            int r1 = min(mu, (pr + 1) * rchunk);
            for (int r = pr * rchunk; r < r1; ++r) rmu = __fma_rn(S.w[r] * YSEL(r, i), YSEL(r, j), rmu);
            part4[pr][ij] = rmu;
        }
    }
    {
        __syncthreads();
        const double hs = S.hs;
        const double decay = 1.0 + c1 * ((1.0 - hs) * cc * (2.0 - cc)) - c1 - cmu;
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            if (j < i) continue;
            double v = 0.0;
            if (!(k.block && (i / k.block != j / k.block))) {
                double rmu = __dadd_rn(__dadd_rn(part4[0][e], part4[1][e]), __dadd_rn(part4[2][e], part4[3][e]));
                v = __dadd_rn(__dadd_rn(__dmul_rn(decay, S.C[e]), __dmul_rn(c1, S.pc[i] * S.pc[j])), __dmul_rn(cmu, rmu));
            }
            part4[0][e] = v;  // the same thread read part4[*][e] above
        }
        __syncthreads();
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            if (j < i) S.A[e] = S.A[j * d + i];
        }
        __syncthreads();
    }
    for (int e = tid; e < dd; e += nt) {
        S.C[e] = S.A[e];
        st->C[e] = S.A[e];
    }
#undef YSEL
    __syncthreads();
    if (!do_sqrt) {
        if (tid == 0) cma_sigma_step(k, st, S.n2, sigma);
        return;
    }
    cma_sqrt_phases<DC>(k, st, S, tid, nt, true, sigma);
}

// C^(1/2) and C^(-1/2) by the coupled Newton-Schulz iteration for the matrix
// square root (Higham, Functions of Matrices, SIAM 2008, Ch. 6): with
// A = C / c, Y_0 = A and Z_0 = I,
//     T_k = (3 I - Z_k Y_k) / 2,   Y_{k+1} = Y_k T_k,   Z_{k+1} = T_k Z_k,
// Y_k -> A^(1/2) and Z_k -> A^(-1/2), quadratically once close, whenever the
// eigenvalues of A lie in (0, 3).  c is the power of two at or above
// max(trace C / d, r / 2.5), r the largest absolute row sum of C (a bound on
// its largest eigenvalue; the target is taken in FP32 with a little margin):
// the eigenvalues land in (0, 2.5], C = I gives A = I, and dividing by c and
// multiplying by sqrt(c) cost no rounding and no FP64 division or square
// root.  Every iterate is a polynomial in C, so FP64 rounding stays at the
// level of the result (no eigenvector step whose errors would freeze in; the
// iterates are not symmetrised: a numpy prototype that mirrored the upper
// triangles of both T and Y, Z diverged from condition number 1e6 on,
// although mirroring either alone converged); the residual of a
// numpy prototype on d = 9 was 3e-15 for condition numbers up to 10, 1e-13
// at 1e3, 1e-10 at 1e6, in 6, 13 and 22 steps (on the GPU: 29 steps and
// 2e-15 at 4e8, where the eigen path's FP32 Jacobi pass no longer resolves
// the small eigenvalues).  The loop stops one step after
// max |I - Z_k Y_k| < 1e-8 (that step squares the residual) and gives up
// after kNsMaxSteps steps (returns false; the caller takes the eigen path and
// later updates keep it until the next reset).  A block-diagonal C keeps
// exactly zero off-diagonal blocks (every product of block-diagonal factors
// has them).  One block; d x d arrays in shared memory: the iterates in S.A
// (d = 9: four fit) or S.A, S.V, S.V2, S.B (d = 18), T in S.A2.
constexpr int kNsMaxSteps = 64;

template <int DC>
__device__ __forceinline__ double ns_dot(const double *L, const double *R, int i, int j)
{
    constexpr int d = DC;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;  // three chains: FP64 latency, not throughput, bounds this
#pragma unroll
    for (int q = 0; q < d; q += 3) {
        a0 = __fma_rn(L[i * d + q], R[q * d + j], a0);
        if (q + 1 < d) a1 = __fma_rn(L[i * d + q + 1], R[(q + 1) * d + j], a1);
        if (q + 2 < d) a2 = __fma_rn(L[i * d + q + 2], R[(q + 2) * d + j], a2);
    }
    return __dadd_rn(__dadd_rn(a0, a1), a2);
}

template <int DC>
__device__ __forceinline__ bool cma_sqrt_newton_schulz(const CmaConst &k, CmaState *st, TellSmem &S, int tid,
                                                       int nt, bool do_sigma, double sigma)
{
    constexpr int d = DC, dd = d * d;
    constexpr bool kPacked = 4 * dd <= kMaxD * kMaxD;
    static_assert(DC > 0 && dd <= kMaxD * kMaxD, "d x d iterates");
    double *Y = S.A, *Z = kPacked ? S.A + dd : S.V, *Y2 = kPacked ? S.A + 2 * dd : S.V2,
           *Z2 = kPacked ? S.A + 3 * dd : S.B, *T = S.A2;
    const double *C = S.C;
    if (tid < 32) {  // the scale c = 2^e, chosen in FP32 (kept in S.part[1][0])
        float tr = 0.0f, row = 0.0f;
        if (tid < d) {
            tr = (float)C[tid * d + tid];
            for (int q = 0; q < d; ++q) row += fabsf((float)C[tid * d + q]);
        }
        for (int o = 16; o; o >>= 1) {
            tr += __shfl_xor_sync(0xffffffffu, tr, o);
            row = fmaxf(row, __shfl_xor_sync(0xffffffffu, row, o));
        }
        if (tid == 0) {
            int e = 0;
            const float m = frexpf(fmaxf(tr / d, 1.0001f * row / 2.5f), &e);  // target = m 2^e, m in [1/2, 1)
            S.part[1][0] = (m > 0.0f) ? (double)e : 0.0;
        }
    }
    __syncthreads();
    const int e2 = (int)S.part[1][0];
    const double ic = ldexp(1.0, -e2);
    // the first step needs no products: Z_0 = I makes Z_0 Y_0 = Y_0 and
    // T_0 Z_0 = T_0 exactly (bit for bit what the products would give)
    bool open0 = false;
    for (int e = tid; e < dd; e += nt) {
        const int i = e / d, j = e - i * d;
        const double y = __dmul_rn(C[e], ic);
        const double r = ((i == j) ? 1.0 : 0.0) - y;
        open0 |= !(fabs(r) < 1e-8);
        const double t = ((i == j) ? 1.0 : 0.0) + 0.5 * r;
        Y[e] = y;
        T[e] = t;
        Z[e] = t;
    }
    bool done = !__syncthreads_or(open0);
    for (int e = tid; e < dd; e += nt) Y2[e] = ns_dot<DC>(Y, T, e / d, e - (e / d) * d);
    __syncthreads();
    {
        double *t = Y; Y = Y2; Y2 = t;
    }
    int steps = 1;
    while (!done && steps < kNsMaxSteps) {
        bool open = false;  // a residual entry at or above 1e-8 (or not a number)
        for (int e = tid; e < dd; e += nt) {
            const int i = e / d, j = e - i * d;
            const double r = ((i == j) ? 1.0 : 0.0) - ns_dot<DC>(Z, Y, i, j);  // I - Z Y
            open |= !(fabs(r) < 1e-8);
            T[e] = ((i == j) ? 1.0 : 0.0) + 0.5 * r;  // (3 I - Z Y) / 2
        }
        done = !__syncthreads_or(open);
        for (int e = tid; e < 2 * dd; e += nt) {
            const int m = e >= dd, f = e - m * dd, i = f / d, j = f - i * d;
            if (m) Z2[f] = ns_dot<DC>(T, Z, i, j);
            else Y2[f] = ns_dot<DC>(Y, T, i, j);
        }
        __syncthreads();
        double *t = Y; Y = Y2; Y2 = t;
        t = Z; Z = Z2; Z2 = t;
        ++steps;
    }
    if (!done) {
        if (tid == 0) atomicOr(&st->warn, 2);
        return false;
    }
    // outputs: C^(1/2) = sqrt(c) Y, C^(-1/2) = Z / sqrt(c) (sqrt(c) a power of
    // two, times sqrt 2 for odd e), symmetrised; the
    // step size on a thread that has no entry (FP64 exp off the critical path)
    const double sc = ldexp((e2 & 1) ? M_SQRT2 : 1.0, e2 >> 1), isc = ldexp((e2 & 1) ? M_SQRT1_2 : 1.0, -(e2 >> 1));
    for (int e = tid; e < dd; e += nt) {
        const int i = e / d, j = e - i * d;
        if (j < i) continue;
        const double h = __dmul_rn(0.5 * __dadd_rn(Y[i * d + j], Y[j * d + i]), sc);
        const double ih = __dmul_rn(0.5 * __dadd_rn(Z[i * d + j], Z[j * d + i]), isc);
        st->C_half[i * d + j] = h;
        st->C_half[j * d + i] = h;
        st->C_half_df[i * d + j] = split_df(h);
        st->C_half_df[j * d + i] = split_df(h);
        st->C_inv_half[i * d + j] = ih;
        st->C_inv_half[j * d + i] = ih;
    }
    if (tid == nt - 1) {
        if (do_sigma) cma_sigma_step(k, st, S.n2, sigma);
        st->jacobi_sweeps = -steps;
    }
    return true;
}

// C^(1/2) and C^(-1/2) of C (held in S.C), with the step-size update when
// do_sigma: the Newton-Schulz iteration, else the eigen path (which also
// stores the eigenbasis, its next warm start).
template <int DC>
__device__ __forceinline__ void cma_sqrt_phases(const CmaConst &k, CmaState *st, TellSmem &S, int tid, int nt,
                                                bool do_sigma, double sigma)
{
    const int d = DC ? DC : k.d, dd = d * d;
    // the Newton-Schulz iteration first (a handful of FP64 matrix products),
    // unless it failed since the last reset
    if constexpr (DC > 0) {
        if (!(st->warn & 2)) {
            if (cma_sqrt_newton_schulz<DC>(k, st, S, tid, nt, do_sigma, sigma)) return;
        }
    }
    for (int e = tid; e < dd; e += nt) S.B[e] = st->B[e];  // the previous basis: the warm start
    __syncthreads();

    // ---- eigendecomposition, phase 1: one-sided (Hestenes) Jacobi in FP32 on
    //      the columns of X = C B (B = last generation's basis, a warm start),
    //      one warp, columns in shared memory.  Each round pairs the columns by
    //      the circle method; a pair (u, w) is rotated by the angle that makes
    //      u . w = 0, cot 2 theta = (|w|^2 - |u|^2) / (2 u . w).  When every
    //      pair has |u . w| <= 1e-5 |u| |w| the columns of C B J are orthogonal
    //      to that level, so B J is an eigenbasis of C up to off-diagonal terms
    //      of V^T C V below 1e-5 of the diagonal, which the FP64 square-root
    //      refinement absorbs (its error is of third order in them).  Column j
    //      of C B J is then lambda_j (B J)_j: with the columns in registers
    //      (d <= 12) the basis is the normalised columns; the shared-memory
    //      form (d = 18) accumulates J alongside ----
    for (int e = tid; e < dd; e += nt) {
        const int i = e / d, j = e - i * d;
        float acc = 0.0f;
        for (int q = 0; q < d; ++q) acc = fmaf((float)S.C[i * d + q], (float)S.B[q * d + j], acc);
        S.Af[j * d + i] = acc;                   // column j of C B
        S.Vf2[j * d + i] = (i == j) ? 1.0f : 0.0f;  // column j of J
    }
    __syncthreads();
    constexpr bool kRegs = DC > 0 && DC <= 12;  // columns in registers, basis from the columns
    if (tid < 32) {
        if constexpr (kRegs)
            onesided_jacobi_regs<DC>(S.Af, tid, st);
        else
            onesided_jacobi_smem<DC>(S.Af, S.Vf2, d, tid, st);
    }
    if (do_sigma && tid == (nt > 32 ? 32 : 0))  // step size (CSA): on the second warp, off the eigendecomposition's critical path
        cma_sigma_step(k, st, S.n2, sigma);
    __syncthreads();
    // ---- phase 2: V = orth(B J) in FP64 (two Newton-Schulz polar steps,
    //      V <- V (3 I - V^T V) / 2, taking 1e-6 to FP64 rounding); B J is the
    //      normalised columns of X (register path) or B times the accumulated J ----
    double *V = S.V, *V2 = S.V2, *A = S.A, *A2 = S.A2;
    if constexpr (kRegs) {
        if (tid < d) {  // 1 / |x_j| for column j
            double n2 = 0.0;
            for (int q = 0; q < d; ++q) n2 = __fma_rn((double)S.Af[tid * d + q], (double)S.Af[tid * d + q], n2);
            S.part[0][tid] = rsqrt(n2);
        }
        __syncthreads();
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            V[e] = (double)S.Af[j * d + i] * S.part[0][j];
        }
    } else {
        for (int e = tid; e < dd; e += nt) {  // J row-major
            const int i = e / d, j = e - i * d;
            S.Vf[e] = S.Vf2[j * d + i];
        }
        __syncthreads();
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            double acc = 0.0;
            for (int q = 0; q < d; ++q) acc = __fma_rn(S.B[i * d + q], (double)S.Vf[q * d + j], acc);
            V[e] = acc;
        }
    }
    __syncthreads();
    for (int step = 0; step < 2; ++step) {
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            double acc = 0.0;
            for (int q = 0; q < d; ++q) acc = __fma_rn(V[q * d + i], V[q * d + j], acc);
            A2[e] = ((i == j) ? 1.5 : 0.0) - 0.5 * acc;
        }
        __syncthreads();
        for (int e = tid; e < dd; e += nt) {
            int i = e / d, j = e - i * d;
            double acc = 0.0;
            for (int q = 0; q < d; ++q) acc = __fma_rn(V[i * d + q], A2[q * d + j], acc);
            V2[e] = acc;
        }
        __syncthreads();
        double *t = V; V = V2; V2 = t;
    }
    sandwich64(d, V, S.C, A2, A, tid, nt);  // A = V^T C V
    // ---- phase 3: C^(1/2) and C^(-1/2) from the near-diagonal A = V^T C V.
    //      A = D + F with F off-diagonal (about 1e-6 of A after the FP32
    //      pass).  Two Newton steps for the square root started from D^(1/2)
    //      give A^(1/2) = S + O(F^3) with S = D^(1/2) + X + Z, where X and Z
    //      solve the Sylvester equations
    //        D^(1/2) X + X D^(1/2) = F,    D^(1/2) Z + Z D^(1/2) = -X^2,
    //      entrywise X_ij = F_ij / (sqrt d_i + sqrt d_j): only sums of
    //      eigenvalues divide, never differences, so clustered eigenvalues
    //      cost nothing.  With W = D^(-1/2) (X + Z), S = D^(1/2) (I + W) and
    //      S^(-1) = (I - W + W^2) D^(-1/2) + O(W^3).  Then C^(1/2) = V S V^T
    //      and C^(-1/2) = V S^(-1) V^T, exact up to the O(F^3) terms because V
    //      is orthogonal to FP64 rounding ----
    if (tid < d) {
        double emax = 0.0;
        for (int i = 0; i < d; ++i) emax = fmax(emax, A[i * d + i]);
        double e = A[tid * d + tid];
        if (!(e > 0.0)) {
            e = fmax(emax, 1e-300) * 1e-14;
            atomicOr(&st->warn, 1);
        }
        st->ev[tid] = e;
        double r = rsqrt(e);
        S.sq[tid] = e * r;
        S.isq[tid] = r;
    }
    __syncthreads();
    double *X = A2, *P = S.C, *Wm = S.B, *W2 = V2;
    for (int e = tid; e < dd; e += nt) {  // X
        const int i = e / d, j = e - i * d;
        X[e] = (i == j) ? 0.0 : A[e] * rcp64(S.sq[i] + S.sq[j]);
    }
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {  // X^2
        const int i = e / d, j = e - i * d;
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = __fma_rn(X[i * d + q], X[q * d + j], acc);
        P[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {  // S (in place of X) and W
        const int i = e / d, j = e - i * d;
        const double y = __fma_rn(-P[e], rcp64(S.sq[i] + S.sq[j]), X[e]);  // X + Z
        Wm[e] = S.isq[i] * y;
        X[e] = (i == j) ? S.sq[i] + y : y;
    }
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {  // W^2
        const int i = e / d, j = e - i * d;
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = __fma_rn(Wm[i * d + q], Wm[q * d + j], acc);
        W2[e] = acc;
    }
    __syncthreads();
    double *Si = S.C;
    for (int e = tid; e < dd; e += nt) {  // S^(-1)
        const int i = e / d, j = e - i * d;
        Si[e] = (((i == j) ? 1.0 : 0.0) - Wm[e] + W2[e]) * S.isq[j];
    }
    __syncthreads();
    double *T1 = A, *T2 = V2;
    for (int e = tid; e < dd; e += nt) {  // V S and V S^(-1)
        const int i = e / d, j = e - i * d;
        double a1 = 0.0, a2 = 0.0;
        for (int q = 0; q < d; ++q) {
            a1 = __fma_rn(V[i * d + q], X[q * d + j], a1);
            a2 = __fma_rn(V[i * d + q], Si[q * d + j], a2);
        }
        T1[e] = a1;
        T2[e] = a2;
    }
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {  // (V S) V^T, (V S^(-1)) V^T; upper triangle mirrored
        const int i = e / d, j = e - i * d;
        if (j < i) continue;
        double h = 0.0, ih = 0.0;
        for (int q = 0; q < d; ++q) {
            h = __fma_rn(T1[i * d + q], V[j * d + q], h);
            ih = __fma_rn(T2[i * d + q], V[j * d + q], ih);
        }
        st->C_half[i * d + j] = h;
        st->C_half[j * d + i] = h;
        st->C_half_df[i * d + j] = split_df(h);
        st->C_half_df[j * d + i] = split_df(h);
        st->C_inv_half[i * d + j] = ih;
        st->C_inv_half[j * d + i] = ih;
    }
    for (int e = tid; e < dd; e += nt) st->B[e] = V[e];
}

static __device__ __noinline__ void cma_tell_block(const CmaConst &k, CmaState *st, const double *y,
                                                   const float *params, const float *loss, TellSmem &S, int tid,
                                                   int nt, bool do_sqrt = true)
{
    if (k.d == 9) cma_tell_impl<9>(k, st, y, params, loss, S, tid, nt, do_sqrt);
    else if (k.d == 18) cma_tell_impl<18>(k, st, y, params, loss, S, tid, nt, do_sqrt);
    else cma_tell_impl<0>(k, st, y, params, loss, S, tid, nt, do_sqrt);
}

// The square roots and eigenbasis of the stored C alone: completes an update
// made with do_sqrt = false (the step size was updated then).
template <int DC>
__device__ __forceinline__ void cma_sqrt_only(const CmaConst &k, CmaState *st, TellSmem &S, int tid, int nt)
{
    const int d = DC ? DC : k.d, dd = d * d;
    for (int e = tid; e < dd; e += nt) {
        S.C[e] = st->C[e];
        S.B[e] = st->B[e];
    }
    __syncthreads();
    cma_sqrt_phases<DC>(k, st, S, tid, nt, false, 0.0);
}

static __device__ __noinline__ void cma_sqrt_block(const CmaConst &k, CmaState *st, TellSmem &S, int tid, int nt)
{
    if (k.d == 9) cma_sqrt_only<9>(k, st, S, tid, nt);
    else if (k.d == 18) cma_sqrt_only<18>(k, st, S, tid, nt);
    else cma_sqrt_only<0>(k, st, S, tid, nt);
}

// Frame epilogue: the frame's best candidate becomes the estimate.
// Joint angle from the unconstrained coordinate (Sec. III-A.3, inverse map).
__device__ __forceinline__ double q_from_qhat(double qh, double lb, double ub)
{
    if (ub == lb) return lb;
    return lb + 0.5 * (ub - lb) * (1.0 - cos(M_PI * (qh - lb) / (ub - lb)));
}

// Is state coordinate i a joint, and which one (0..2)?
__device__ __forceinline__ int joint_of(int i) { const int r = i % 9; return r >= 6 ? r - 6 : -1; }

// Kalman prediction s <- F s, P <- F P F^T + Q (F = [[1, dt], [0, 1]] per coordinate).
__device__ __forceinline__ void kf_predict(const KfConst &c, KfState &f, int i)
{
    const double dt = c.dt;
    double *s = f.s[i], *P = f.P[i];
    s[0] += dt * s[1];
    const double p00 = P[0] + 2.0 * dt * P[1] + dt * dt * P[2] + c.q_pos[i];
    const double p01 = P[1] + dt * P[2];
    P[0] = p00;
    P[1] = p01;
    P[2] = P[2] + c.q_vel[i];
}

// The filter's position of coordinate i back in state units (joint angles
// clamped to their limits, then mapped to the unconstrained coordinate).
__device__ __forceinline__ double kf_to_state(const CmaConst &k, const KfState &f, int i)
{
    const int j = joint_of(i);
    const double x = f.s[i][0];
    if (j < 0) return x;
    const double q = fmin(k.q_ub[j], fmax(k.q_lb[j], x));
    return qhat_from_q(q, k.q_lb[j], k.q_ub[j]);
}

// Frame epilogue: the frame's best candidate becomes the estimate; with the
// filter on it is the measurement z_t of the Kalman update (joints as angles)
// and the filtered state becomes the estimate.
__device__ __forceinline__ void cma_finish_frame(const CmaConst &k, CmaState *st, float *pose_out, int tid, int nt)
{
    const bool kf = k.kf.enabled != 0;
    const bool first = kf && !st->kf.initialized;
    for (int i = tid; i < k.d; i += nt) {
        const float b = st->best_x[i];
        double e = (double)b;
        if (kf) {
            const int j = joint_of(i);
            const double z = j < 0 ? e : q_from_qhat(e, k.q_lb[j], k.q_ub[j]);
            KfState &f = st->kf;
            double *s = f.s[i], *P = f.P[i];
            if (first) {
                s[0] = z;
                s[1] = 0.0;
                P[0] = k.kf.r[i];
                P[1] = 0.0;
                P[2] = k.kf.p_vel0[i];
            } else {  // gain K = P H^T / (H P H^T + r), H = [1 0]
                const double S = P[0] + k.kf.r[i];
                const double k0 = P[0] / S, k1 = P[1] / S, y = z - s[0];
                s[0] += k0 * y;
                s[1] += k1 * y;
                const double p00 = (1.0 - k0) * P[0], p01 = (1.0 - k0) * P[1], p11 = P[2] - k1 * P[1];
                P[0] = p00;
                P[1] = p01;
                P[2] = p11;
            }
            e = kf_to_state(k, f, i);
        }
        st->est[i] = e;
        if (pose_out) pose_out[i] = kf ? (float)e : b;
    }
    __syncthreads();
    if (first && tid == 0) st->kf.initialized = 1;
}

}  // namespace trk
