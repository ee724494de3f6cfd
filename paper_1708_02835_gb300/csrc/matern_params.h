/*
 * Per-launch constants of the Matern covariance generator (Eq. 2).  Filled on
 * the host by egs_matern_params_init (matern_host.c) and read by the device
 * kernels in matern.cuh.  Plain C so both gcc and nvcc compile it.
 */
#ifndef EGS_MATERN_PARAMS_H
#define EGS_MATERN_PARAMS_H

#define EGS_TEMME_MAX 24 /* terms of Temme's series (x <= 1.25) */
#define EGS_CF_MAX 140   /* depth of the backward recurrence (x > 1.25) */
#define EGS_EXP_TAB 64   /* entries of the exponential's table (2^(j/64)) */

/* Local polynomials of theta1^-1 e^x C(x) for general nu (built on the device
 * per evaluation, matern.cu): x / 1.25 in [2^E0, 2^(E0 + OCT)), each octave
 * cut into SUB equal sub-intervals, NC monomial coefficients each in the
 * local variable s in [-1, 1). */
#define EGS_MT_OCT 22
#define EGS_MT_SUB 8
#define EGS_MT_NC 12
#define EGS_MT_E0 (-12)
#define EGS_MT_DOUBLES (EGS_MT_OCT * EGS_MT_SUB * EGS_MT_NC)
/* device scratch of a mixed-precision evaluation's generator: the FP64
 * polynomials, then the same split into float pairs */
#define EGS_MT_SCRATCH_DOUBLES (2 * EGS_MT_DOUBLES)

/* distance between two locations */
#define EGS_DIST_EUCLIDEAN 0    /* (x, y) in the plane */
#define EGS_DIST_GREAT_CIRCLE 1 /* (longitude, latitude) in degrees, haversine */
#define EGS_EARTH_RADIUS_KM 6371.0

/* kind of covariance evaluation */
#define EGS_MATERN_GENERAL 0 /* any theta3: Temme / backward recurrence */
#define EGS_MATERN_HALF 1    /* theta3 = 1/2: theta1 exp(-x) */
#define EGS_MATERN_3HALF 2   /* theta3 = 3/2: theta1 (1 + x) exp(-x) */
#define EGS_MATERN_5HALF 3   /* theta3 = 5/2: theta1 (1 + x + x^2/3) exp(-x) */

typedef struct {
    double th1, th2, inv_th2, nu, mu;
    double c;      /* theta1 / (2^(nu-1) Gamma(nu)) */
    double two_mu; /* 2^mu */
    double fact;   /* mu pi / sin(mu pi), 1 at mu = 0 */
    double g1;     /* Gamma_1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu) */
    double g2;     /* Gamma_2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2 */
    double gp;     /* Gamma(1 + mu) */
    double gm;     /* Gamma(1 - mu) */
    int kind;
    int N;         /* nu = mu + N */
    int half_mu;   /* |mu| = 1/2: C_k = 0 for k >= 1, the recurrence is not needed */
    int metric;    /* EGS_DIST_EUCLIDEAN or EGS_DIST_GREAT_CIRCLE */
    double radius; /* sphere radius of the great-circle distance */
    double t_k2[EGS_TEMME_MAX + 1]; /* 1 / (k^2 - mu^2) */
    double t_km[EGS_TEMME_MAX + 1]; /* 1 / (k - mu) */
    double t_kp[EGS_TEMME_MAX + 1]; /* 1 / (k + mu) */
    double t_k[EGS_TEMME_MAX + 1];  /* 1 / k */
    double cf_q[EGS_CF_MAX + 2];    /* (k + 1/2)^2 - mu^2 */
    double cf_c[EGS_CF_MAX + 2];    /* C_k = prod_{j=1..k} ((j - 1/2)^2 - mu^2) / j, C_0 = 1 */
    double cf_ic[EGS_CF_MAX + 2];   /* 1 / C_k (unused when half_mu) */
    double exp_tab[EGS_EXP_TAB];    /* theta1 2^(-j/64), j = 0..63: the table of theta1 e^-x */
} egs_matern_params;

/* Constants of the double-float evaluation of the closed-form kinds
 * (matern_df.cuh): 1/theta2 and the table theta1 2^(-j/256), j = 0..255, each
 * as a float pair (hi, lo). */
#define EGS_DF_TAB 256
typedef struct {
    float inv_th2[2];
    int kind;
    int pad;
    float tab[2 * EGS_DF_TAB]; /* hi at 2j, lo at 2j + 1 */
} egs_matern_df;

#ifdef __cplusplus
extern "C" {
#endif
/* Returns 0 on success, -1 if theta is not finite and positive. */
int egs_matern_params_init(const double theta[3], egs_matern_params *P);
/* Fills D for the double-float path; returns 0 if that path applies
 * (theta1 and 1/theta2 well inside the float range), -1 if not. */
int egs_matern_df_init(const egs_matern_params *P, egs_matern_df *D);
#ifdef __cplusplus
}
#endif

#endif
