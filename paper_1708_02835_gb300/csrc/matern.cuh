// Device evaluation of the Matern covariance, Eq. 2 (Section 2.2):
//   C(r) = theta1 / (2^(nu-1) Gamma(nu)) x^nu K_nu(x),  x = r / theta2,  nu = theta3,
// with C(0) = theta1 (the limit x^nu K_nu(x) -> 2^(nu-1) Gamma(nu), DLMF 10.30.2).
//
// Half-integer smoothness has closed forms (Section 2.2 names nu = 1/2, the
// exponential model; nu = 3/2 and 5/2 follow from K_{n+1/2}, DLMF 10.39.2 and
// 10.49.12).  Any other nu is evaluated as nu = mu + N, |mu| <= 1/2:
//   x <= 1.25: Temme's series for K_mu and K_{mu+1};
//   x >  1.25: Miller's backward recurrence for the minimal solution of the
//              confluent hypergeometric recurrence, giving e^x K_mu and
//              e^x K_{mu+1} (Temme 1975; Thompson & Barnett 1986);
//   then N steps of K_{m+1} = K_{m-1} + (2m/x) K_m.
// The loop lengths are made warp-uniform (the maximum over the active lanes),
// so the per-k constants, staged in shared memory, are read as broadcasts.
#pragma once
#include <cuda_runtime.h>

#include "matern_params.h"

namespace egs {

__device__ __forceinline__ int warp_max_active(int v)
{
    return __reduce_max_sync(__activemask(), v);
}

// Terms of Temme's series needed for ~1e-17 truncation at x <= 1.25.
__device__ __forceinline__ int temme_terms(double x)
{
    return x <= 0.1 ? 8 : (x <= 0.5 ? 12 : 16);
}

// Depth of the backward recurrence for full double accuracy at x > 1.25.
__device__ __forceinline__ int cf_depth(double x)
{
    int k = (int)(14.0 + 152.0 / x) + 1;
    return k > EGS_CF_MAX ? EGS_CF_MAX : k;
}

// x^nu K_nu(x) * c for the general case, x > 0 (times e^x if scaled: the
// table builder's form, finite up to x of a few thousand).
// Pp points to the constants staged in shared memory.
__device__ __forceinline__ double matern_general(const egs_matern_params *__restrict__ Pp, double x,
                                                 bool scaled = false)
{
    const egs_matern_params &P = *Pp;
    const double mu = P.mu;
    double kmu, kmu1;  // K_mu, K_{mu+1}   (scaled by e^x in the recurrence branch)
    double front;      // c * x^nu (times e^-x in the recurrence branch)
    if (x <= 1.25) {
        // Temme's series.  lx = log(2/x), sigma = mu lx.
        const double lx = -log(0.5 * x);
        const double sig = mu * lx;
        const double es = exp(sig);  // (2/x)^mu
        const double ies = 1.0 / es; // (x/2)^mu
        const double ch = 0.5 * (es + ies);
        double shs;                  // sinh(sigma) / sigma
        if (fabs(sig) < 0.1) {
            const double s2 = sig * sig;
            shs = 1.0 + s2 / 6.0 * (1.0 + s2 / 20.0 * (1.0 + s2 / 42.0 * (1.0 + s2 / 72.0)));
        } else {
            shs = 0.5 * (es - ies) / sig;
        }
        double f = P.fact * (ch * P.g1 + shs * lx * P.g2);
        double p = 0.5 * es * P.gp;
        double q = 0.5 * ies * P.gm;
        const double d = 0.25 * x * x;
        double ck = 1.0;
        double s0 = f, s1 = p;
        const int nt = warp_max_active(temme_terms(x));
        for (int k = 1; k <= nt; ++k) {
            const double kd = (double)k;
            f = (kd * f + p + q) * P.t_k2[k];
            p *= P.t_km[k];
            q *= P.t_kp[k];
            ck *= d * P.t_k[k];
            s0 = fma(ck, f, s0);
            s1 = fma(ck, p - kd * f, s1);
        }
        kmu = s0;
        kmu1 = s1 * 2.0 / x;
        // x^nu = x^N * 2^mu * (x/2)^mu
        double xn = 1.0;
        for (int j = 0; j < P.N; ++j) xn *= x;
        front = P.c * P.two_mu * ies * xn;
        if (scaled) front *= exp(x);
    } else {
        // Backward recurrence z_{k-1} = 2(k + x) z_k - q_k z_{k+1}, z_{K+1} = 0,
        // accumulating s = sum_k C_k z_k; S = s / z_0 and z_1 / z_0 are
        // independent of the starting scale.  The start z_K = 1 / C_K keeps
        // s near 1; every 8 steps all three are rescaled by 2^-512 when they
        // grow past 2^512 (exact, so the ratios are unchanged).
        double S = 1.0, r1 = 0.0;
        if (!P.half_mu) {
            const int K = warp_max_active(cf_depth(x));
            const double x2 = 2.0 * x;
            double zk1 = 0.0, zk = P.cf_ic[K];
            double s = 1.0;
            for (int k = K; k >= 1; --k) {
                const double zm1 = fma(2.0 * (double)k + x2, zk, -P.cf_q[k] * zk1);
                zk1 = zk;
                zk = zm1;
                s = fma(P.cf_c[k - 1], zk, s);
                if ((k & 7) == 0 && fmax(fabs(zk), fabs(s)) > 0x1p512) {
                    zk *= 0x1p-512;
                    zk1 *= 0x1p-512;
                    s *= 0x1p-512;
                }
            }
            const double inv_z0 = 1.0 / zk;
            S = s * inv_z0;
            r1 = zk1 * inv_z0;
        }
        // e^x K_mu = sqrt(pi / (2x)) / S
        kmu = 1.2533141373155002512 * rsqrt(x) / S;
        kmu1 = kmu * (mu + x + 0.5 - (0.25 - mu * mu) * r1) / x;
        front = P.c * exp(scaled ? P.nu * log(x) : P.nu * log(x) - x);
    }
    double knu = kmu;
    if (P.N >= 1) {
        double km = kmu, kc = kmu1;
        const double ix = 1.0 / x;
        for (int j = 1; j < P.N; ++j) {
            const double kn = fma(2.0 * (mu + (double)j) * ix, kc, km);
            km = kc;
            kc = kn;
        }
        knu = kc;
    }
    return front * knu;
}

// Distance between locations i and j.  Euclidean: sqrt(dx^2 + dy^2).  Great
// circle (Section 7.4): the haversine formula on (longitude, latitude) in
// degrees, hav(d / R) = hav(phi_j - phi_i) + cos(phi_i) cos(phi_j)
// hav(lambda_j - lambda_i), hav(t) = sin^2(t / 2), d = 2 R asin(sqrt(hav)).
__device__ __forceinline__ double loc_dist(const egs_matern_params *__restrict__ Pp, double xi, double yi, double xj,
                                           double yj)
{
    if (Pp->metric == EGS_DIST_EUCLIDEAN) {
        const double dx = xi - xj, dy = yi - yj;
        return sqrt(fma(dx, dx, dy * dy));
    }
    const double rad = 0.017453292519943295769;  // pi / 180
    const double p1 = yi * rad, p2 = yj * rad;
    const double s1 = sin(0.5 * (p2 - p1)), s2 = sin(0.5 * (xj - xi) * rad);
    const double h = fma(cos(p1) * cos(p2), s2 * s2, s1 * s1);
    return 2.0 * Pp->radius * asin(sqrt(fmin(h, 1.0)));
}

// theta1 e^-x for x >= 0 by the table-driven method of P. T. P. Tang ("Table-
// driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM Trans. Math. Softw. 15, 1989): with k = rint(64 x / ln 2),
// m = k >> 6, j = k & 63 and r = x - k ln2/64 (|r| <= ln2/128, Cody-Waite
// reduction with a 36-bit high part of ln2/64, exact for k < 2^17),
//   theta1 e^-x = 2^-m (theta1 2^(-j/64)) e^-r,
// the table entry from the host (binary128, rounded once), e^-r - 1 by its
// Taylor polynomial of degree 5 (truncation below 4e-17), and 2^-m applied to
// the exponent field with integer operations.  About 10 FP64 operations,
// within about one ulp; values below the smallest normal double give 0.
__device__ __forceinline__ double th1_exp_neg(const egs_matern_params *__restrict__ Pp, double x)
{
    if (!(x < 708.0)) return x == x ? 0.0 : x;  // e^-708 is near the smallest normal; NaN stays NaN
    constexpr double kInvLn2_64 = 92.332482616893656877;   // 64 / ln 2
    constexpr double kShift = 6755399441055744.0;          // 1.5 * 2^52
    constexpr double kLn2_64_hi = 0x1.62e42fefa0000p-7;    // ln2/64, 36 significant bits
    constexpr double kLn2_64_lo = 0x1.cf79abc9e3b3ap-46;   // ln2/64 - kLn2_64_hi
    const double t = fma(x, kInvLn2_64, kShift);           // k in the low bits of t
    const double kd = t - kShift;
    const int k = __double2loint(t);
    double r = fma(-kd, kLn2_64_hi, x);
    r = fma(-kd, kLn2_64_lo, r);
    const double u = -r;
    double p = fma(u, 1.0 / 120.0, 1.0 / 24.0);
    p = fma(u, p, 1.0 / 6.0);
    p = fma(u, p, 0.5);
    p = fma(u, p, 1.0);
    p *= u;                                                // e^u - 1
    const double tj = Pp->exp_tab[k & (EGS_EXP_TAB - 1)];
    const double v = fma(tj, p, tj);
    const long long bits = __double_as_longlong(v);
    const int m = k >> 6;
    if ((int)((bits >> 52) & 0x7FF) - m <= 0) return 0.0;
    return __longlong_as_double(bits - ((long long)m << 52));
}

// Smallest x covered by the local polynomials (below it: Temme's series).
constexpr double kMtXlo = 1.25 * 0x1p-12;

// C(x) for general nu from the local polynomials (x in [kMtXlo, 708)): with
// y = x / 1.25 = 2^e (1 + (j + (1 + s) / 2) / 8), e the octave and j the
// sub-interval (both read from the bits of y), s in [-1, 1) is formed from
// the remaining mantissa bits without rounding; C = p_{e,j}(s) theta1 e^-x.
// About 25 FP64 operations.
__device__ __forceinline__ double matern_table_eval(const egs_matern_params *__restrict__ Pp,
                                                    const double *__restrict__ tab, double x)
{
    const double y = x * 0.8;
    const long long yb = __double_as_longlong(y);
    const int oct = (int)((yb >> 52) & 0x7FF) - 1023 - EGS_MT_E0;
    const int iv = oct * EGS_MT_SUB + (int)((yb >> 49) & 7);
    const double v = __longlong_as_double(((yb & 0x1FFFFFFFFFFFFll) << 3) | 0x3FF0000000000000ll);
    const double s = fma(2.0, v, -3.0);
    const double *a = tab + iv * EGS_MT_NC;
    double p = a[EGS_MT_NC - 1];
#pragma unroll
    for (int j = EGS_MT_NC - 2; j >= 0; --j) p = fma(p, s, a[j]);
    return p * th1_exp_neg(Pp, x);
}

// C(x * theta2) for x = r / theta2 >= 0.  tab: the local polynomials of a
// general nu (shared or global memory), or NULL for the direct evaluation.
__device__ __forceinline__ double matern_eval(const egs_matern_params *__restrict__ Pp, double x,
                                              const double *__restrict__ tab = nullptr)
{
    const egs_matern_params &P = *Pp;
    if (x == 0.0) return P.th1;
    switch (P.kind) {
    case EGS_MATERN_HALF: return th1_exp_neg(Pp, x);
    case EGS_MATERN_3HALF: return (1.0 + x) * th1_exp_neg(Pp, x);
    case EGS_MATERN_5HALF: return fma(x, fma(x, 1.0 / 3.0, 1.0), 1.0) * th1_exp_neg(Pp, x);
    default:
        if (tab && x >= kMtXlo) return x < 708.0 ? matern_table_eval(Pp, tab, x) : (x == x ? 0.0 : x);
        return matern_general(Pp, x);
    }
}

// One warp builds the local polynomial of sub-interval iv (0 <= iv <
// EGS_MT_OCT * EGS_MT_SUB): lanes 0..NC-1 evaluate g = theta1^-1 e^x C(x) at
// the NC Chebyshev points of the interval with the direct method, lane 0
// forms the Chebyshev coefficients c_k = (2 / NC) sum_i g_i cos(pi k (i + 1/2) / NC)
// (c_0 halved) and converts sum_k c_k T_k(s) to monomials in s (T_{k+1} =
// 2 s T_k - T_{k-1}).  vals: NC doubles of shared memory for this warp.
__device__ __forceinline__ void matern_table_interval(const egs_matern_params *__restrict__ Pp, int iv, double *tab,
                                                      double *vals)
{
    const int lane = threadIdx.x & 31;
    const int oct = iv / EGS_MT_SUB, sub = iv % EGS_MT_SUB;
    if (lane < EGS_MT_NC) {
        const double t = cospi((2.0 * lane + 1.0) / (2.0 * EGS_MT_NC));  // Chebyshev point in s
        const double y = ldexp(1.0 + (sub + 0.5 * (1.0 + t)) / EGS_MT_SUB, oct + EGS_MT_E0);
        const double x = 1.25 * y;
        vals[lane] = matern_general(Pp, x, true) / Pp->th1;
    }
    __syncwarp();
    if (lane == 0) {
        double c[EGS_MT_NC], a[EGS_MT_NC], tkm[EGS_MT_NC], tk[EGS_MT_NC], tn[EGS_MT_NC];
        for (int k = 0; k < EGS_MT_NC; ++k) {
            double acc = 0.0;
            for (int i = 0; i < EGS_MT_NC; ++i) acc = fma(vals[i], cospi(k * (2.0 * i + 1.0) / (2.0 * EGS_MT_NC)), acc);
            c[k] = acc * (k == 0 ? 1.0 : 2.0) / EGS_MT_NC;
            a[k] = 0.0;
            tkm[k] = tk[k] = 0.0;
        }
        tkm[0] = 1.0;  // T_0
        tk[1] = 1.0;   // T_1
        a[0] = c[0];
        a[1] = c[1];
        for (int k = 1; k + 1 < EGS_MT_NC; ++k) {
            // T_{k+1} = 2 s T_k - T_{k-1}
            for (int j = 0; j < EGS_MT_NC; ++j) tn[j] = (j > 0 ? 2.0 * tk[j - 1] : 0.0) - tkm[j];
            for (int j = 0; j < EGS_MT_NC; ++j) {
                a[j] = fma(c[k + 1], tn[j], a[j]);
                tkm[j] = tk[j];
                tk[j] = tn[j];
            }
        }
        for (int j = 0; j < EGS_MT_NC; ++j) tab[iv * EGS_MT_NC + j] = a[j];
    }
    __syncwarp();
}

}  // namespace egs
