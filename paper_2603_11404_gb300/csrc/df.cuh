// Double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and FMA-based TwoProd
// (Dekker 1971 / Ogita-Rump-Oishi 2005); add, multiply, divide and square root
// follow Dekker's double-length algorithms.  Explicit _rn intrinsics keep the
// compiler from contracting the transformations.  GB300 runs FP32 FMA at 128
// lanes/clk/SM against ~1.6 FP64 FMA/clk/SM, so this is how the library gets
// near-FP64 accuracy for the per-candidate kinematics.
//
// sin/cos: Cody-Waite reduction by pi/2 split into a float with few bits (so
// n * P1 is exact) and a double-float remainder, then the Taylor series of sin
// and cos on [-pi/4, pi/4] to the 17th / 18th power, evaluated by Estrin's
// scheme (independent pairs, then the powers u^2, u^4, u^8).
#pragma once

#include <math.h>

namespace trk {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_from(float a) { return {a, 0.0f}; }

__device__ __forceinline__ dfl quick_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_sum_df(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfl two_prod_df(float a, float b)
{
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = two_sum_df(a.hi, b.hi);
    dfl t = two_sum_df(a.lo, b.lo);
    float e = __fadd_rn(s.lo, t.hi);
    dfl u = quick_two_sum(s.hi, e);
    return quick_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    dfl p = two_prod_df(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p.hi, e);
}

__device__ __forceinline__ dfl df_mul_f(dfl a, float b)
{
    dfl p = two_prod_df(a.hi, b);
    return quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a * b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) { return df_add(df_mul(a, b), c); }

__device__ __forceinline__ dfl df_div(dfl a, dfl b)
{
    float q1 = __fdiv_rn(a.hi, b.hi);
    dfl r = df_sub(a, df_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul_f(b, q2));
    float q3 = __fdiv_rn(r.hi, b.hi);
    return df_add(quick_two_sum(q1, q2), df_from(q3));
}

__device__ __forceinline__ dfl df_sqrt(dfl a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    float s = __fsqrt_rn(a.hi);
    dfl e = df_sub(a, two_prod_df(s, s));
    return quick_two_sum(s, __fdiv_rn(e.hi, __fmul_rn(2.0f, s)));
}

// hi/lo split of a double done by the compiler (constant expressions only).
#define DFL_CONST(x) dfl{(float)(x), (float)((x) - (double)(float)(x))}

// Taylor coefficients (-1)^j/(2j+1)! and (-1)^j/(2j)! as double-float
// constants folded into the instructions (no constant-bank loads: the first
// evaluation in a CTA would otherwise wait on constant-cache misses).
#define TS0 DFL_CONST(1.0)
#define TS1 DFL_CONST(-1.0 / 6.0)
#define TS2 DFL_CONST(1.0 / 120.0)
#define TS3 DFL_CONST(-1.0 / 5040.0)
#define TS4 DFL_CONST(1.0 / 362880.0)
#define TS5 DFL_CONST(-1.0 / 39916800.0)
#define TS6 DFL_CONST(1.0 / 6227020800.0)
#define TS7 DFL_CONST(-1.0 / 1307674368000.0)
#define TS8 DFL_CONST(1.0 / 355687428096000.0)
#define TC0 DFL_CONST(1.0)
#define TC1 DFL_CONST(-1.0 / 2.0)
#define TC2 DFL_CONST(1.0 / 24.0)
#define TC3 DFL_CONST(-1.0 / 720.0)
#define TC4 DFL_CONST(1.0 / 40320.0)
#define TC5 DFL_CONST(-1.0 / 3628800.0)
#define TC6 DFL_CONST(1.0 / 479001600.0)
#define TC7 DFL_CONST(-1.0 / 87178291200.0)
#define TC8 DFL_CONST(1.0 / 20922789888000.0)
#define TC9 DFL_CONST(-1.0 / 6402373705728000.0)

struct dfl2 {
    dfl s, c;
};

// sin and cos of a double-float angle (|x| up to ~1e4 keeps the reduction
// exact).  Kept out of line and with rolled loops: it is called from several
// places once per candidate, so compact code matters more than a few cycles.
static __device__ __noinline__ dfl2 df_sincos(dfl x)
{
    // pi/2 = P1 + P2 with P1 = 201/128 (8 significant bits) and P2 a double-float
    const float P1 = 1.5703125f;
    const dfl P2 = DFL_CONST(1.5707963267948966 - 1.5703125);
    const float n = rintf(__fmul_rn(x.hi, 0.636619772f));
    dfl r = df_sub(x, df_from(__fmul_rn(n, P1)));  // n * P1 exact for |n| < 2^15
    r = df_sub(r, df_mul_f(P2, n));
    const dfl u = df_mul(r, r);
    // sin r = r * S(u), S(u) = sum_{j=0..8} s_j u^j;  cos r = C(u) = sum_{j=0..9} c_j u^j,
    // u = r^2, evaluated by Estrin's scheme (independent pairs, then powers
    // u^2, u^4, u^8) to keep the dependent chain short
    const dfl u2 = df_mul(u, u), u4 = df_mul(u2, u2), u8 = df_mul(u4, u4);
    dfl s01 = df_fma(TS1, u, TS0), s23 = df_fma(TS3, u, TS2);
    dfl s45 = df_fma(TS5, u, TS4), s67 = df_fma(TS7, u, TS6);
    dfl c01 = df_fma(TC1, u, TC0), c23 = df_fma(TC3, u, TC2);
    dfl c45 = df_fma(TC5, u, TC4), c67 = df_fma(TC7, u, TC6), c89 = df_fma(TC9, u, TC8);
    dfl s03 = df_fma(s23, u2, s01), s47 = df_fma(s67, u2, s45);
    dfl c03 = df_fma(c23, u2, c01), c47 = df_fma(c67, u2, c45);
    dfl ps = df_fma(TS8, u8, df_fma(s47, u4, s03));
    dfl pc = df_fma(c89, u8, df_fma(c47, u4, c03));
    dfl sr = df_mul(ps, r);
    dfl cr = pc;
    int q = ((int)n) & 3;
    dfl ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
    if (q == 1 || q == 2) cc = df_neg(cc);  // cos: +c, -s, -c, +s
    if (q >= 2) ss = df_neg(ss);            // sin: +s, +c, -s, -c
    return {ss, cc};
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace trk
