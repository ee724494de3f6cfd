// Matern covariance (Eq. 2) for the half-integer smoothness values that have
// closed forms (nu = 1/2, 3/2, 5/2), evaluated in double-float arithmetic:
// every quantity is an unevaluated sum h + l of two floats, |l| <= ulp(h)/2,
// which carries about 48 significant bits.  GB300 issues FP32 (and INT32)
// operations 64 times faster than FP64 ones, so ~130 single-precision
// operations per entry cost a fraction of the ~28 FP64 operations of the
// direct evaluation; the result is accurate to about 1e-14 relative, enough
// for the mixed precisions (FP32 storage of the off-band tiles, and the
// refinement residual, which regenerates Sigma while it multiplies).
//
// Building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (FastTwoSum; TwoProduct, here by one fused multiply-add), and the
// double-word algorithms of Joldes, Muller & Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic" (ACM
// TOMS 44, 2017).  The square root takes one Newton correction in the style
// of Karp & Markstein (ACM TOMS 23, 1997) from the correctly rounded float
// root.  e^-x follows Tang's table-driven method (ACM TOMS 15, 1989) with a
// 256-entry table, so that the correction polynomial only needs its leading
// term in double-float.
#pragma once
#include <cuda_runtime.h>

#include "matern.cuh"
#include "matern_params.h"

namespace egs {
namespace df {

struct F2 {
    float h, l;
};

// a + b exactly (Knuth): s + e = a + b.
__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b exactly when a == 0 or exponent(a) >= exponent(b) (Dekker).
__device__ __forceinline__ F2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b exactly: p + e with e from one fused multiply-add.
__device__ __forceinline__ F2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Double-word sum (the "sloppy" algorithm: accurate when the operands do not
// nearly cancel, which holds wherever it is used below: positive operands,
// or |y| much smaller than |x|).
__device__ __forceinline__ F2 add(F2 x, F2 y)
{
    const F2 s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(__fadd_rn(s.l, x.l), y.l));
}

// Double-word product (DWTimesDW of Joldes et al., relative error < 5 u^2).
__device__ __forceinline__ F2 mul(F2 x, F2 y)
{
    F2 p = two_prod(x.h, y.h);
    const float t = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h));
    return fast_two_sum(p.h, __fadd_rn(p.l, t));
}

// x^2 for a double word.
__device__ __forceinline__ F2 sqr(F2 x)
{
    F2 p = two_prod(x.h, x.h);
    return fast_two_sum(p.h, __fmaf_rn(__fmul_rn(2.0f, x.h), x.l, p.l));
}

// sqrt(x) for x >= 0: the correctly rounded float root s, then
// s + (x - s^2) / (2 s) with the residual x - s^2 formed exactly by one fused
// multiply-add (|correction| <= ulp(s) / 2, so 1 / (2 s) is needed to float
// accuracy only).
__device__ __forceinline__ F2 sqrt_df(F2 x)
{
    if (x.h <= 0.0f) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(x.h);
    const float r = __fadd_rn(__fmaf_rn(-s, s, x.h), x.l);
    return fast_two_sum(s, __fmul_rn(r, __fmul_rn(0.5f, __frsqrt_rn(x.h))));
}

// x_i - x_j for coordinates split as h + l (a float pair per coordinate).
__device__ __forceinline__ F2 diff(float ih, float il, float jh, float jl)
{
    const F2 a = two_sum(ih, -jh);
    return two_sum(a.h, __fadd_rn(a.l, __fsub_rn(il, jl)));
}

// Per-evaluation constants (built on the host, matern_host.c).
struct Consts {
    F2 inv_th2;  // 1 / theta2
    int kind;    // EGS_MATERN_HALF / 3HALF / 5HALF / GENERAL
};

// theta1 e^-x for a double-word x >= 0 by Tang's method: k = rint(256 x /
// ln 2), m = k >> 8, j = k & 255, r = x - k ln2/256 (|r| <= ln2/512, the
// constant ln2/256 split into three floats c1 + c2 + c3 with c1 carrying 8
// significant bits, so that k c1 is exact for k < 2^16, and k c2 exact as a
// product pair); then theta1 e^-x = 2^-m T_j (1 + p), T_j = theta1 2^(-j/256)
// from the double-word table tab (hi at 2j, lo at 2j + 1) and
// p = u + u^2 (1/2 + u/6 + u^2/24), u = -r (|u^5/120| < 4e-17).  Values of x
// beyond 150 (e^-150 < 1e-65) give 0.
__device__ __forceinline__ F2 th1_exp_neg_df(F2 x, const float *__restrict__ tab)
{
    if (!(x.h < 150.0f)) return {0.0f, 0.0f};
    constexpr float kInvC = 369.32993f;       // 256 / ln 2, any nearby float works (k is only a reduction index)
    constexpr float kShift = 12582912.0f;     // 1.5 * 2^23
    constexpr float c1 = 0x1.62p-9f;          // ln2/256 to 8 bits (the bits beyond are in c2 + c3)
    constexpr float c2 = 0x1.c85fep-18f;      // ln2/256 - c1 rounded to float
    constexpr float c3 = -0x1.718432p-43f;    // ln2/256 - c1 - c2 rounded to float (rest 4e-21)
    const float t = __fmaf_rn(x.h, kInvC, kShift);
    const float kf = __fsub_rn(t, kShift);
    const int k = __float_as_int(t) - __float_as_int(kShift);
    const float a = __fmaf_rn(-kf, c1, x.h);  // exact (see above)
    const F2 p2 = two_prod(kf, c2);
    const F2 s = two_sum(a, -p2.h);
    const float lo = __fadd_rn(s.l, __fmaf_rn(-kf, c3, __fsub_rn(x.l, p2.l)));
    const F2 r = fast_two_sum(s.h, lo);
    const F2 u{-r.h, -r.l};
    // v = u^2 (1/2 + wq), wq = u/6 + u^2/24: 1/2 is exact, so wq needs only
    // float accuracy (|u^2 wq| < 5e-10)
    const float wq = __fmul_rn(u.h, __fmaf_rn(u.h, 1.0f / 24.0f, 1.0f / 6.0f));
    const F2 u2 = sqr(u);
    const F2 v = fast_two_sum(__fmul_rn(0.5f, u2.h), __fmaf_rn(u2.h, wq, __fmul_rn(0.5f, u2.l)));
    const F2 p = add(u, v);                   // e^u - 1
    const int j = k & 255;
    const F2 T{tab[2 * j], tab[2 * j + 1]};
    F2 w = two_prod(T.h, p.h);
    w.l = __fmaf_rn(T.h, p.l, __fmaf_rn(T.l, p.h, w.l));
    const F2 s2 = fast_two_sum(T.h, w.h);     // |w| < |T| / 700
    F2 res = fast_two_sum(s2.h, __fadd_rn(__fadd_rn(s2.l, T.l), w.l));
    // 2^-m in two exact power-of-two factors (m <= 217), so that results
    // below the float range underflow gradually instead of wrapping
    const int m = k >> 8;
    const int m1 = m < 120 ? m : 120;
    const float f1 = __int_as_float((127 - m1) << 23);
    const float f2 = __int_as_float((127 - (m - m1)) << 23);
    res.h = __fmul_rn(__fmul_rn(res.h, f1), f2);
    res.l = __fmul_rn(__fmul_rn(res.l, f1), f2);
    return res;
}

// C(r) for r given by the double-word squared distance r2 (Eq. 2 with the
// closed forms: nu = 1/2 theta1 e^-x; 3/2 theta1 (1 + x) e^-x; 5/2
// theta1 (1 + x + x^2 / 3) e^-x; x = r / theta2).
__device__ __forceinline__ F2 matern_closed_df(const Consts &C, F2 x, const float *__restrict__ tab)
{
    F2 e = th1_exp_neg_df(x, tab);
    if (C.kind == EGS_MATERN_3HALF) {
        e = mul(e, add(F2{1.0f, 0.0f}, x));
    } else if (C.kind == EGS_MATERN_5HALF) {
        const F2 x2 = sqr(x);
        const F2 third = mul(x2, F2{0x1.555556p-2f, -0x1.555556p-27f});  // x^2 / 3
        e = mul(e, add(add(F2{1.0f, 0.0f}, x), third));
    }
    return e;
}

// p * s + a for double words (Horner step).
__device__ __forceinline__ F2 mul_add(F2 p, F2 s, F2 a)
{
    F2 m = two_prod(p.h, s.h);
    m.l = __fmaf_rn(p.h, s.l, __fmaf_rn(p.l, s.h, m.l));
    const F2 t = two_sum(m.h, a.h);
    return fast_two_sum(t.h, __fadd_rn(__fadd_rn(t.l, m.l), a.l));
}

// C(x) for a general nu from the local polynomials of g(x) = theta1^-1 e^x C(x)
// (built per evaluation in FP64 on the device and split into float pairs,
// ctab[iv * EGS_MT_NC + j] = coefficient j of sub-interval iv): y = x / 1.25
// = 2^e (1 + (sub + (1 + s) / 2) / 8), the octave e and sub-interval sub read
// from the bits of y's high part, s = 16 (y - centre) / 2^e exact in double
// words (the centre shares y's binade); then p(s) by Horner's rule -- the
// terms of degree >= 6 in float, where the coefficients have decayed below
// 1e-8 of the constant term (the expansion converges like 34^-j: every
// sub-interval lies 17 half-widths from the branch point at 0) -- and
// C = p(s) theta1 e^-x.  Valid for x in [1.25 2^EGS_MT_E0, 1.25 2^(EGS_MT_E0 +
// EGS_MT_OCT)); the caller handles smaller x.
__device__ __forceinline__ F2 matern_table_df(F2 x, const float2 *__restrict__ ctab, const float *__restrict__ etab)
{
    const F2 y = mul(x, F2{0x1.99999ap-1f, -0x1.99999ap-27f});  // 0.8 (residual 2^-52)
    const unsigned yb = __float_as_uint(y.h);
    const int e = (int)(yb >> 23) - 127;
    const int sub = (int)((yb >> 20) & 7u);
    const int iv = (e - EGS_MT_E0) * EGS_MT_SUB + sub;
    const float centre = __uint_as_float((yb & 0xFF800000u) | ((unsigned)sub << 20) | 0x80000u);
    const float scale = __uint_as_float((unsigned)(127 + 4 - e) << 23);  // 16 / 2^e
    const F2 sv = two_sum(__fmul_rn(__fsub_rn(y.h, centre), scale), __fmul_rn(y.l, scale));
    const float2 *a = ctab + iv * EGS_MT_NC;
    float q = a[EGS_MT_NC - 1].x;
#pragma unroll
    for (int j = EGS_MT_NC - 2; j >= 6; --j) q = __fmaf_rn(q, sv.h, a[j].x);
    F2 pv{q, 0.0f};
#pragma unroll
    for (int j = 5; j >= 0; --j) pv = mul_add(pv, sv, F2{a[j].x, a[j].y});
    return mul(pv, th1_exp_neg_df(x, etab));
}

// One off-diagonal entry (i != j) of Sigma from the split coordinates
// (xh, xl, yh, yl) of both locations.  GENERAL: the local polynomials ctab;
// the rare x below their range (near-duplicate locations) takes Temme's
// series in FP64 from the direct evaluation's constants P.
template <bool GENERAL>
__device__ __forceinline__ F2 matern_entry_df(const Consts &C, const float4 &pi, const float4 &pj,
                                              const float *__restrict__ etab, const float2 *__restrict__ ctab,
                                              const egs_matern_params *__restrict__ P)
{
    const F2 dx = diff(pi.x, pi.y, pj.x, pj.y);
    const F2 dy = diff(pi.z, pi.w, pj.z, pj.w);
    const F2 x = mul(sqrt_df(add(sqr(dx), sqr(dy))), C.inv_th2);
    if (!GENERAL) return matern_closed_df(C, x, etab);
    if (!(x.h < 150.0f)) return {0.0f, 0.0f};
    if (x.h >= 1.0001f * (float)kMtXlo) return matern_table_df(x, ctab, etab);
    const double v = matern_eval(P, (double)x.h + (double)x.l, nullptr);
    const float vh = __double2float_rn(v);
    return {vh, __double2float_rn(v - (double)vh)};
}

}  // namespace df
}  // namespace egs
