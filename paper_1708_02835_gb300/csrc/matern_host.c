/*
 * Per-launch constants of the Matern generator (Eq. 2), computed once on the
 * host in IEEE binary128 (_Float128) so that the device kernels only run
 * short recurrences per matrix entry.
 *
 * The device evaluates K_nu with nu = mu + N, |mu| <= 1/2, N >= 0 an integer:
 *  - x <= 1.25: Temme's series (N. M. Temme, "On the numerical evaluation of the
 *    modified Bessel function of the third kind", J. Comput. Phys. 19, 1975).
 *    It needs Gamma_1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu),
 *    Gamma_2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2, Gamma(1 +- mu) and
 *    mu pi / sin(mu pi).
 *  - x > 1.25: Miller's backward recurrence for the minimal solution
 *    z_k = U(mu + 1/2 + k, 2 mu + 1, 2x) of the confluent hypergeometric
 *    three-term recurrence in the first parameter (DLMF 13.3.7), normalised by
 *    sum_k C_k z_k = (2x)^(-mu-1/2) (the continued-fraction approach of
 *    Temme 1975 and Thompson & Barnett, J. Comput. Phys. 64, 1986).  It needs
 *    q_k = (k + 1/2)^2 - mu^2 and C_k = prod_{j<=k} ((j - 1/2)^2 - mu^2) / j.
 *  - N upward steps of K_{m+1} = K_{m-1} + (2m/x) K_m (DLMF 10.29.1).
 * The Matern prefactor theta1 / (2^(nu-1) Gamma(nu)) is formed here as well,
 * and the table theta1 2^(-j/64), j = 0..63, of the device's table-driven
 * exponential (matern.cuh).
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <string.h>

#include "matern_params.h"

typedef _Float128 q_t;

static const q_t Q_PI = 3.141592653589793238462643383279502884f128;
static const q_t Q_EULER = 0.577215664901532860606512090082402431f128;

int egs_matern_params_init(const double theta[3], egs_matern_params *P)
{
    memset(P, 0, sizeof(*P));
    for (int i = 0; i < 3; ++i)
        if (!isfinite(theta[i]) || !(theta[i] > 0.0)) return -1;
    double nu = theta[2];
    P->th1 = theta[0];
    P->th2 = theta[1];
    P->inv_th2 = 1.0 / theta[1];
    P->nu = nu;
    if (nu == 0.5) P->kind = EGS_MATERN_HALF;
    else if (nu == 1.5) P->kind = EGS_MATERN_3HALF;
    else if (nu == 2.5) P->kind = EGS_MATERN_5HALF;
    else P->kind = EGS_MATERN_GENERAL;

    int N = (int)floor(nu + 0.5);
    double mu = nu - (double)N; /* exact: Sterbenz */
    if (mu >= 0.5) { mu -= 1.0; N += 1; }
    P->N = N;
    P->mu = mu;

    q_t qnu = (q_t)nu, qmu = (q_t)mu;
    q_t c = (q_t)theta[0] / (powf128(2.0f128, qnu - 1.0f128) * tgammaf128(qnu));
    P->c = (double)c;
    P->two_mu = (double)powf128(2.0f128, qmu);

    q_t gp = tgammaf128(1.0f128 + qmu), gm = tgammaf128(1.0f128 - qmu);
    P->gp = (double)gp;
    P->gm = (double)gm;
    P->g2 = (double)((1.0f128 / gm + 1.0f128 / gp) * 0.5f128);
    if (fabs(mu) < 1e-13) {
        /* Gamma_1(mu) = -gamma_E + O(mu^2); the O(mu^2) term is below 1e-26 here */
        P->g1 = (double)(-Q_EULER);
        P->fact = 1.0;
    } else {
        P->g1 = (double)((1.0f128 / gm - 1.0f128 / gp) / (2.0f128 * qmu));
        P->fact = (double)(Q_PI * qmu / sinf128(Q_PI * qmu));
    }

    for (int k = 1; k <= EGS_TEMME_MAX; ++k) {
        q_t qk = (q_t)k;
        P->t_k2[k] = (double)(1.0f128 / (qk * qk - qmu * qmu));
        P->t_km[k] = (double)(1.0f128 / (qk - qmu));
        P->t_kp[k] = (double)(1.0f128 / (qk + qmu));
        P->t_k[k] = (double)(1.0f128 / qk);
    }
    q_t C = 1.0f128;
    P->cf_c[0] = 1.0;
    P->cf_ic[0] = 1.0;
    P->half_mu = (fabs(mu) == 0.5);
    for (int k = 1; k <= EGS_CF_MAX + 1; ++k) {
        q_t qk = (q_t)k;
        q_t h = qk - 0.5f128;
        C = C * (h * h - qmu * qmu) / qk;
        P->cf_c[k] = (double)C;
        P->cf_ic[k] = (C != 0.0f128) ? (double)(1.0f128 / C) : 0.0;
        q_t g = qk + 0.5f128;
        P->cf_q[k] = (double)(g * g - qmu * qmu);
    }
    q_t g0 = 0.5f128;
    P->cf_q[0] = (double)(g0 * g0 - qmu * qmu);
    /* theta1 2^(-j/64) for the table-driven exponential of the half-integer kinds */
    for (int j = 0; j < EGS_EXP_TAB; ++j)
        P->exp_tab[j] = (double)((q_t)theta[0] * exp2f128(-(q_t)j / (q_t)EGS_EXP_TAB));
    return 0;
}

/* The double-float constants: q rounded to a float pair (hi, lo). */
static void split_q(q_t q, float *hi, float *lo)
{
    const float h = (float)q;
    *hi = h;
    *lo = (float)(q - (q_t)h);
}

int egs_matern_df_init(const egs_matern_params *P, egs_matern_df *D)
{
    memset(D, 0, sizeof(*D));
    /* theta1 2^(-j/256) and its low part must stay normal floats down to the
     * smallest table entry; 1/theta2 likewise */
    const double lim = 0x1p60;
    if (!(P->th1 > 1.0 / lim && P->th1 < lim && P->inv_th2 > 1.0 / lim && P->inv_th2 < lim)) return -1;
    D->kind = P->kind;
    split_q(1.0f128 / (q_t)P->th2, &D->inv_th2[0], &D->inv_th2[1]);
    for (int j = 0; j < EGS_DF_TAB; ++j)
        split_q((q_t)P->th1 * exp2f128(-(q_t)j / (q_t)EGS_DF_TAB), &D->tab[2 * j], &D->tab[2 * j + 1]);
    return 0;
}
