// Device-side CMA-ES building blocks (arXiv 2603.11404, Sec. III-A.1,
// Eq. cmaes_update; block-diagonal form of Sec. III-B), shared by the
// stand-alone CMA-ES kernels and the fused per-generation fitness kernel.
//
// Precision plan (GB300's FP64 pipe is narrow and slow: a dependent FP64 FMA
// costs ~64 cycles, division and square root ~700): the covariance, paths and
// step size are FP64; sampling draws FP32 normals; the eigendecomposition runs
// a warm-started FP32 Jacobi pass for the bulk of the rotation, then makes the
// basis orthogonal in FP64 (Newton-Schulz) and finishes with FP64 Jacobi
// sweeps whose rotation angles come from FP32 formulas and whose (c, s) pairs
// are re-normalised in FP64, so the result is accurate to FP64 rounding
// without FP64 divisions or square roots in the inner loop.
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
    float Af[kMaxD * kMaxD], Af2[kMaxD * kMaxD], Vf[kMaxD * kMaxD], Vf2[kMaxD * kMaxD];
    float rc[kMaxD / 2 + 1], rs[kMaxD / 2 + 1];
    double rcd[kMaxD / 2 + 1], rsd[kMaxD / 2 + 1];
    int rp[kMaxD / 2 + 1], rq[kMaxD / 2 + 1];
    double n2, hs;
};

// Jacobi rotation (c, s) in FP32 that annihilates a_pq of the 2x2 block
// [[a_pp, a_pq], [a_pq, a_qq]] (Golub & Van Loan, symmetric Schur
// decomposition); diff = a_qq - a_pp is formed by the caller in the matrix's
// own precision so that near-equal diagonals keep their difference.
__device__ __forceinline__ void jacobi_angle_f32(float diff, float apq, float &c, float &s)
{
    if (apq == 0.0f) {
        c = 1.0f;
        s = 0.0f;
        return;
    }
    // approximate intrinsics suffice: the rotation only has to be close to the
    // annihilating one (the FP64 sweeps finish the job and re-normalise (c, s))
    float tau = __fdividef(diff, 2.0f * apq);
    float t;
    if (fabsf(tau) > 1e18f) {
        t = __fdividef(0.5f, tau);
    } else {
        float h = 1.0f + tau * tau;
        t = __fdividef(1.0f, fabsf(tau) + h * rsqrtf(h));
    }
    if (tau < 0.0f) t = -t;
    if (!isfinite(t)) t = 0.0f;
    c = rsqrtf(1.0f + t * t);
    s = t * c;
}

// Pair `pr` of round s of the round-robin (circle) ordering on n2 indices.
__device__ __forceinline__ void rr_pair(int n2, int s, int pr, int &p, int &q)
{
    if (pr == 0) {
        p = n2 - 1;
        q = s;
    } else {
        p = (s + pr) % (n2 - 1);
        q = (s - pr + (n2 - 1)) % (n2 - 1);
    }
}

// A' = J^T A J and V' = V J for one round of disjoint rotations (pairs of
// indices rp/rq with cosines rc/rs); indices >= d are padding.  Templated on
// the precision; every thread of the block calls it.
template <typename T>
__device__ __forceinline__ void jacobi_round_apply(int d, int np, const int *rp, const int *rq, const T *rc,
                                                   const T *rs, const T *A, T *A2, const T *V, T *V2, int tid, int nt)
{
    // consecutive items go to different warps, so a block of several warps
    // spreads the work over all of its sub-partitions' pipes
    if (nt > 32 && nt % 32 == 0) tid = (tid & 31) * (nt >> 5) + (tid >> 5);
    for (int e = tid; e < np * np; e += nt) {  // 2x2 block (P, Q)
        int P = e / np, Q = e - P * np;
        int ip[2] = {rp[P], rq[P]}, jq[2] = {rp[Q], rq[Q]};
        T cP = rc[P], sP = rs[P], cQ = rc[Q], sQ = rs[Q];
        T M[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) M[a][b] = (ip[a] < d && jq[b] < d) ? A[ip[a] * d + jq[b]] : (T)0;
        T t0[2], t1[2];
        for (int a = 0; a < 2; ++a) {
            t0[a] = cQ * M[a][0] - sQ * M[a][1];
            t1[a] = sQ * M[a][0] + cQ * M[a][1];
        }
        T o00 = cP * t0[0] - sP * t0[1], o10 = sP * t0[0] + cP * t0[1];
        T o01 = cP * t1[0] - sP * t1[1], o11 = sP * t1[0] + cP * t1[1];
        if (ip[0] < d && jq[0] < d) A2[ip[0] * d + jq[0]] = o00;
        if (ip[1] < d && jq[0] < d) A2[ip[1] * d + jq[0]] = o10;
        if (ip[0] < d && jq[1] < d) A2[ip[0] * d + jq[1]] = o01;
        if (ip[1] < d && jq[1] < d) A2[ip[1] * d + jq[1]] = o11;
    }
    for (int e = tid; e < d * np; e += nt) {  // V J
        int i = e / np, P = e - i * np;
        int p = rp[P], q = rq[P];
        T c = rc[P], s = rs[P];
        if (p < d && q < d) {
            T vp = V[i * d + p], vq = V[i * d + q];
            V2[i * d + p] = c * vp - s * vq;
            V2[i * d + q] = s * vp + c * vq;
        } else {
            int r = (p < d) ? p : q;
            if (r < d) V2[i * d + r] = V[i * d + r];
        }
    }
}

// C (d x d, FP64, row-major) -> out = X^T C X for square X, FP64.
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

// The whole update from the fitness of the last population (called by every
// thread of one block).  y [lam*d] are the FP64 steps of that population.
// DC is the dimension as a compile-time constant (0 = read k.d at run time):
// the index arithmetic below divides by d and by the number of Jacobi pairs,
// which is cheap only for constant divisors.
template <int DC>
__device__ __forceinline__ void cma_tell_impl(const CmaConst &k, CmaState *st, const double *y, const float *params,
                                              const float *loss, TellSmem &S, int tid, int nt)
{
    const int d = DC ? DC : k.d, lam = k.lam, dd = d * d, mu = k.mu;
    for (int i = tid; i < lam; i += nt) {
        float v = loss[i];
        S.sl[i] = isnan(v) ? INFINITY : v;
    }
    for (int e = tid; e < dd; e += nt) {
        S.C[e] = st->C[e];
        S.B[e] = st->B[e];
        S.A2[e] = st->C_inv_half[e];
    }
    for (int r = tid; r < mu; r += nt) S.w[r] = k.w[r];
    __syncthreads();
    // stable ranking by (loss, index)
    for (int i = tid; i < lam; i += nt) {
        float li = S.sl[i];
        int r = 0;
        for (int j = 0; j < lam; ++j) {
            float lj = S.sl[j];
            r += (lj < li) || (lj == li && j < i);
        }
        S.order[r] = i;
    }
    __syncthreads();
    if (tid == 0) {
        int b = S.order[0];
        if (S.sl[b] < st->best_loss) {
            st->best_loss = S.sl[b];
            for (int i = 0; i < d; ++i) st->best_x[i] = params[(size_t)b * d + i];
        }
    }
    // the selected steps y_{r:lam}, r < mu, staged in shared memory when they fit
    const bool staged = mu * d <= kYselCap;
    if (staged)
        for (int e = tid; e < mu * d; e += nt) {
            int r = e / d, i = e - r * d;
            S.ysel[e] = y[(size_t)S.order[r] * d + i];
        }
    __syncthreads();
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
    if (tid < d) {
        double acc = 0.0;
        for (int p = 0; p < 8; ++p) acc = __dadd_rn(acc, S.part[p][tid]);
        S.yw[tid] = acc;
    }
    __syncthreads();
    const double sigma = st->sigma, cs = k.c_sigma, cc = k.c_c;
    if (tid < d) {
        double t = 0.0;
        for (int j = 0; j < d; ++j) t = __fma_rn(S.A2[tid * d + j], S.yw[j], t);
        double ps = __dadd_rn(__dmul_rn(1.0 - cs, st->p_sigma[tid]), __dmul_rn(k.ps_coef, t));
        st->p_sigma[tid] = ps;
        S.part[0][tid] = ps * ps;
        double mn = __dadd_rn(st->m[tid], __dmul_rn(k.c_m * sigma, S.yw[tid]));
        st->m[tid] = mn;
        st->m_df[tid] = split_df(mn);
    }
    __syncthreads();
    if (tid == 0) {
        double n2 = 0.0;
        for (int i = 0; i < d; ++i) n2 += S.part[0][i];
        // h_sigma: |p_sigma| / sqrt(1 - (1 - c_sigma)^(2(g+1))) < (1.4 + 2/(n+1)) chi_n, compared squared
        double pw = st->cs_pow * (1.0 - cs) * (1.0 - cs);
        S.n2 = n2;
        S.hs = (n2 < k.hs_thr2 * (1.0 - pw)) ? 1.0 : 0.0;
        st->cs_pow = pw;
    }
    __syncthreads();
    const double hs = S.hs;
    if (tid < d) {
        double v = __dadd_rn(__dmul_rn(1.0 - cc, st->p_c[tid]), __dmul_rn(hs * k.pc_coef, S.yw[tid]));
        st->p_c[tid] = v;
        S.pc[tid] = v;
    }
    __syncthreads();
    // C <- decay C + c1 p_c p_c^T + c_mu sum w_r y_r y_r^T (block form: zero off-diagonal
    // blocks); the rank-mu sum runs as 4 deterministic partial chains held in
    // the (still unused) A, A2, V, V2 buffers
    const double c1 = k.c_1, cmu = k.c_mu;
    const double decay = 1.0 + c1 * ((1.0 - hs) * cc * (2.0 - cc)) - c1 - cmu;
    {
        double *part4[4] = {S.A, S.A2, S.V, S.V2};
        const int rchunk = (mu + 3) / 4;
        for (int e = tid; e < 4 * dd; e += nt) {
            int pr = e / dd, ij = e - pr * dd, i = ij / d, j = ij - i * d;
            if (j < i) continue;
            double rmu = 0.0;
            int r1 = min(mu, (pr + 1) * rchunk);
            for (int r = pr * rchunk; r < r1; ++r) rmu = __fma_rn(S.w[r] * YSEL(r, i), YSEL(r, j), rmu);
            part4[pr][ij] = rmu;
        }
        __syncthreads();
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
    if (tid == 0) {
        double sg = sigma * exp(k.cs_over_ds * (sqrt(S.n2) * k.inv_chi - 1.0));
        st->sigma = sg;
        st->sigma_df = split_df(sg);
        st->gen += 1;
        st->gen_total += 1;
    }
    __syncthreads();

    // ---- eigendecomposition, phase 1: FP32 Jacobi on B^T C B, warm start ----
    const int n2r = d + (d & 1), np = n2r / 2;
    for (int e = tid; e < dd; e += nt) {
        int i = e / d, j = e - i * d;
        float acc = 0.0f;
        for (int q = 0; q < d; ++q) acc = fmaf((float)S.C[i * d + q], (float)S.B[q * d + j], acc);
        S.Af2[e] = acc;
        S.Vf[e] = (i == j) ? 1.0f : 0.0f;
    }
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {
        int i = e / d, j = e - i * d;
        float acc = 0.0f;
        for (int q = 0; q < d; ++q) acc = fmaf((float)S.B[q * d + i], S.Af2[q * d + j], acc);
        S.Af[e] = acc;
    }
    __syncthreads();
    {
        float *Af = S.Af, *Af2 = S.Af2, *Vf = S.Vf, *Vf2 = S.Vf2;
        for (int sweep = 0; sweep < 10; ++sweep) {
            // until the off-diagonal is at FP32 rounding level (relative 1e-6, or
            // 4e-7 of the largest diagonal entry): the FP64 sweep finishes the job
            float amax = 0.0f;
            for (int i = 0; i < d; ++i) amax = fmaxf(amax, fabsf(Af[i * d + i]));
            const float floor2 = (4e-7f * amax) * (4e-7f * amax);
            int off = 0;
            for (int e = tid; e < dd; e += nt) {
                int i = e / d, j = e - i * d;
                if (j > i && Af[e] * Af[e] > 1e-12f * fabsf(Af[i * d + i] * Af[j * d + j]) + floor2) off = 1;
            }
            if (!__syncthreads_or(off)) break;
            for (int s2 = 0; s2 < n2r - 1; ++s2) {
                if (tid < np) {
                    int p, q;
                    rr_pair(n2r, s2, tid, p, q);
                    float c = 1.0f, sn = 0.0f;
                    if (p < d && q < d) jacobi_angle_f32(Af[q * d + q] - Af[p * d + p], Af[p * d + q], c, sn);
                    S.rp[tid] = p;
                    S.rq[tid] = q;
                    S.rc[tid] = c;
                    S.rs[tid] = sn;
                }
                __syncthreads();
                jacobi_round_apply<float>(d, np, S.rp, S.rq, S.rc, S.rs, Af, Af2, Vf, Vf2, tid, nt);
                __syncthreads();
                float *t = Af; Af = Af2; Af2 = t;
                t = Vf; Vf = Vf2; Vf2 = t;
            }
        }
        if (Vf != S.Vf)  // an odd number of rounds left the basis in S.Vf2
            for (int e = tid; e < dd; e += nt) S.Vf[e] = S.Vf2[e];
    }
    __syncthreads();
    const float *Vf = S.Vf;
    // ---- phase 2: V = orth(B Vf) in FP64 (two Newton-Schulz polar steps,
    //      V <- V (3 I - V^T V) / 2, taking 1e-6 to FP64 rounding) ----
    double *V = S.V, *V2 = S.V2, *A = S.A, *A2 = S.A2;
    for (int e = tid; e < dd; e += nt) {
        int i = e / d, j = e - i * d;
        double acc = 0.0;
        for (int q = 0; q < d; ++q) acc = __fma_rn(S.B[i * d + q], (double)Vf[q * d + j], acc);
        V[e] = acc;
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
    // ---- phase 3: FP64 Jacobi sweeps (FP32 angles, FP64-normalised rotations).
    //      The FP32 pass left off-diagonals at ~1e-6 relative; each rotation
    //      removes all but ~1e-7 of its entry, and the cross terms a sweep
    //      leaves are of order off^2 / gap (quadratic convergence), so one sweep
    //      usually reaches ~1e-12.  Clustered eigenvalues (small gaps, common
    //      while C is still near a multiple of I) can leave ~1e-9; a further
    //      sweep runs while any off-diagonal entry exceeds 1e-11 of the largest
    //      diagonal one (at most three sweeps in all) ----
    int sweeps64 = 0;
    for (; sweeps64 < 3; ++sweeps64) {
        if (sweeps64 > 0) {
            double amax = 0.0;
            for (int i = 0; i < d; ++i) amax = fmax(amax, fabs(A[i * d + i]));
            const double tol = 1e-11 * amax;
            int off = 0;
            for (int e = tid; e < dd; e += nt) {
                int i = e / d, j = e - i * d;
                if (j > i && fabs(A[e]) > tol) off = 1;
            }
            if (!__syncthreads_or(off)) break;
        }
        for (int s = 0; s < n2r - 1; ++s) {
            if (tid < np) {
                int p, q;
                rr_pair(n2r, s, tid, p, q);
                double c = 1.0, sn = 0.0;
                if (p < d && q < d && A[p * d + q] != 0.0) {
                    float cf, sf;
                    jacobi_angle_f32((float)(A[q * d + q] - A[p * d + p]), (float)A[p * d + q], cf, sf);
                    double cd = cf, sd = sf;
                    double f = 1.5 - 0.5 * (cd * cd + sd * sd);  // one Newton step to c^2 + s^2 = 1
                    c = cd * f;
                    sn = sd * f;
                }
                S.rp[tid] = p;
                S.rq[tid] = q;
                S.rcd[tid] = c;
                S.rsd[tid] = sn;
            }
            __syncthreads();
            jacobi_round_apply<double>(d, np, S.rp, S.rq, S.rcd, S.rsd, A, A2, V, V2, tid, nt);
            __syncthreads();
            double *t = A; A = A2; A2 = t;
            t = V; V = V2; V2 = t;
        }
    }
    // ---- eigenvalues (clamped positive), basis, C^(1/2), C^(-1/2) ----
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
    if (tid == 0) st->jacobi_sweeps = sweeps64;
    __syncthreads();
    for (int e = tid; e < dd; e += nt) {
        int i = e / d, j = e - i * d;
        double h = 0.0, ih = 0.0;
        for (int q = 0; q < d; ++q) {
            double vv = V[i * d + q] * V[j * d + q];
            h = __fma_rn(vv, S.sq[q], h);
            ih = __fma_rn(vv, S.isq[q], ih);
        }
        st->C_half[e] = h;
        st->C_half_df[e] = split_df(h);
        st->C_inv_half[e] = ih;
        st->B[e] = V[e];
    }
}

static __device__ __noinline__ void cma_tell_block(const CmaConst &k, CmaState *st, const double *y,
                                                   const float *params, const float *loss, TellSmem &S, int tid,
                                                   int nt)
{
    if (k.d == 9) cma_tell_impl<9>(k, st, y, params, loss, S, tid, nt);
    else if (k.d == 18) cma_tell_impl<18>(k, st, y, params, loss, S, tid, nt);
    else cma_tell_impl<0>(k, st, y, params, loss, S, tid, nt);
}

// Frame epilogue: the frame's best candidate becomes the estimate.
__device__ __forceinline__ void cma_finish_frame(const CmaConst &k, CmaState *st, float *pose_out, int tid, int nt)
{
    for (int i = tid; i < k.d; i += nt) {
        float b = st->best_x[i];
        st->est[i] = (double)b;
        if (pose_out) pose_out[i] = b;
    }
}

}  // namespace trk
