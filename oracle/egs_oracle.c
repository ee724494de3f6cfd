/*
 * Plain FP64 CPU oracle for the exact Gaussian log-likelihood with a Matern
 * covariance.  TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and
 * the benchmark's CPU-baseline leg call it; the library's product path never
 * does.  It shares no code with the CUDA path.
 *
 * What it computes, and the passage each function follows:
 *   ora_bessel_k    K_nu(x), the modified Bessel function of the second kind
 *                   that appears in Eq. 2 (Section 2.2).  The paper does not
 *                   say how to evaluate it; this file uses the integral
 *                   representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *                   (DLMF 10.32.9) with the trapezoidal rule, which converges
 *                   geometrically for this even, analytic, doubly-exponentially
 *                   decaying integrand.
 *   ora_matern      Eq. 2: C(r) = th1 / (2^(th3-1) Gamma(th3)) (r/th2)^th3 K_th3(r/th2),
 *                   with C(0) = th1 (the r -> 0 limit, DLMF 10.30.2).
 *   ora_cov_matrix  Sigma_ij = C(||s_i - s_j||) over all i, j (Section 2,
 *                   definition of Sigma; Algorithm 2, genCovMatrix).
 *   ora_cholesky    Sigma = L L^T, textbook column-by-column (left-looking)
 *                   Cholesky (Algorithm 2, dpotrf); a pivot <= 0 reports the
 *                   failing column.
 *   ora_forward_solve  L y = Z (Algorithm 2, dtrsm; the text of Section 6.5
 *                   states the solve as L Z_new = Z_old).
 *   ora_loglik      Eq. 1 through Algorithm 2:
 *                   l = -n/2 log(2 pi) - sum_i log L_ii - 1/2 y^T y,
 *                   log|Sigma| = 2 sum_i log L_ii (the "product of the diagonal
 *                   entries" of the factor in Section 6.1, taken in log form).
 *   ora_brute_*     Brute-force checks in long double: determinant by LU with
 *                   partial pivoting, Z^T Sigma^-1 Z by a Gauss-Jordan inverse.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* e^x K_nu(x) = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt, trapezoidal rule.
 * cosh t - 1 is formed as 2 sinh^2(t/2) to avoid cancellation near t = 0.
 * The step keeps at least ~5 points per standard deviation of the Gaussian-like
 * peak (width 1/sqrt(x)) for large x.  Summation stops past the integrand's
 * maximum once a term is below 1e-22 of the largest term seen. */
double ora_bessel_k_scaled(double nu, double x, double h)
{
    if (!(x > 0.0)) return INFINITY;
    nu = fabs(nu);
    if (h <= 0.0) h = 0.05;
    double hx = 0.2 / sqrt(x);
    if (hx < h) h = hx;
    double t_peak = asinh(nu / x);
    double f0 = 1.0; /* integrand at t = 0 */
    double sum = 0.5 * f0, maxterm = f0;
    for (long k = 1; k < 4000000; ++k) {
        double t = (double)k * h;
        double s = sinh(0.5 * t);
        double term = exp(-x * 2.0 * s * s) * cosh(nu * t);
        sum += term;
        if (term > maxterm) maxterm = term;
        if (t > t_peak && term < 1e-22 * maxterm) break;
    }
    return h * sum;
}

double ora_bessel_k(double nu, double x)
{
    return exp(-x) * ora_bessel_k_scaled(nu, x, 0.05);
}

/* Eq. 2. */
double ora_matern(const double theta[3], double r)
{
    double th1 = theta[0], th2 = theta[1], nu = theta[2];
    if (r == 0.0) return th1;
    double x = r / th2;
    double c = th1 / (pow(2.0, nu - 1.0) * tgamma(nu));
    double ks = ora_bessel_k_scaled(nu, x, 0.05);   /* e^x K_nu(x) */
    return c * exp(nu * log(x) - x) * ks;
}

/* Sigma, dense n x n row-major, both triangles. */
void ora_cov_matrix(int64_t n, const double *x, const double *y, const double theta[3], double *S)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double dx = x[i] - x[j], dy = y[i] - y[j];
            double r = sqrt(dx * dx + dy * dy);
            double c = ora_matern(theta, r);
            S[i * n + j] = c;
            S[j * n + i] = c;
        }
    }
}

/* Sigma_12: rows are the m points (x1, y1), columns the n points (x2, y2). */
void ora_cov_cross(int64_t m, const double *x1, const double *y1, int64_t n, const double *x2,
                   const double *y2, const double theta[3], double *S)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double dx = x1[i] - x2[j], dy = y1[i] - y2[j];
            S[i * n + j] = ora_matern(theta, sqrt(dx * dx + dy * dy));
        }
}

/* In place on the lower triangle of a row-major n x n matrix.  Returns -1 on
 * success, else the column whose pivot was not positive.  The strict upper
 * triangle is set to zero so the result is L itself. */
int64_t ora_cholesky(int64_t n, double *A)
{
    for (int64_t j = 0; j < n; ++j) {
        const double *Lj = A + j * n;
        double d = Lj[j];
        for (int64_t k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
        if (!(d > 0.0)) return j;
        double ljj = sqrt(d);
        A[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double *Li = A + i * n;
            double s = Li[j];
            for (int64_t k = 0; k < j; ++k) s -= Li[k] * Lj[k];
            Li[j] = s / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
    return -1;
}

void ora_forward_solve(int64_t n, const double *L, const double *z, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = z[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
}

/* Algorithm 2 end to end.  Returns -1 on success or the failing column.
 * out[0] = l, out[1] = log|Sigma|, out[2] = Z^T Sigma^-1 Z. */
int64_t ora_loglik(int64_t n, const double *x, const double *y, const double *z, const double theta[3],
                   double out[3])
{
    double *S = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!S || !w) { free(S); free(w); return -2; }
    ora_cov_matrix(n, x, y, theta, S);
    int64_t fail = ora_cholesky(n, S);
    if (fail >= 0) {
        out[0] = out[1] = out[2] = NAN;
        free(S); free(w);
        return fail;
    }
    ora_forward_solve(n, S, z, w);
    double logdet = 0.0, quad = 0.0;
    for (int64_t i = 0; i < n; ++i) logdet += log(S[i * n + i]);
    logdet *= 2.0;
    for (int64_t i = 0; i < n; ++i) quad += w[i] * w[i];
    out[0] = -0.5 * quad - 0.5 * logdet - 0.5 * (double)n * log(2.0 * M_PI);
    out[1] = logdet;
    out[2] = quad;
    free(S); free(w);
    return -1;
}

/* log|det S| by LU with partial pivoting in long double.  Returns the sign of
 * the determinant (+1, -1) or 0 when a pivot is exactly zero. */
int ora_brute_logdet(int64_t n, const double *S, long double *logabsdet)
{
    long double *A = (long double *)malloc(sizeof(long double) * (size_t)n * (size_t)n);
    if (!A) return 0;
    for (int64_t i = 0; i < n * n; ++i) A[i] = S[i];
    int sign = 1;
    long double acc = 0.0L;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabsl(A[i * n + k]) > fabsl(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0L) { free(A); return 0; }
        if (p != k) {
            for (int64_t j = 0; j < n; ++j) {
                long double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            sign = -sign;
        }
        long double piv = A[k * n + k];
        if (piv < 0) sign = -sign;
        acc += logl(fabsl(piv));
        for (int64_t i = k + 1; i < n; ++i) {
            long double f = A[i * n + k] / piv;
            for (int64_t j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
        }
    }
    *logabsdet = acc;
    free(A);
    return sign;
}

/* Z^T S^-1 Z with S^-1 formed by Gauss-Jordan elimination with partial
 * pivoting in long double.  Returns 0 on success, -1 if S is singular. */
int ora_brute_quad(int64_t n, const double *S, const double *z, long double *quad)
{
    int64_t w = 2 * n;
    long double *M = (long double *)malloc(sizeof(long double) * (size_t)n * (size_t)w);
    if (!M) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < w; ++j)
            M[i * w + j] = (j < n) ? (long double)S[i * n + j] : (long double)((j - n) == i);
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabsl(M[i * w + k]) > fabsl(M[p * w + k])) p = i;
        if (M[p * w + k] == 0.0L) { free(M); return -1; }
        if (p != k)
            for (int64_t j = 0; j < w; ++j) {
                long double t = M[k * w + j]; M[k * w + j] = M[p * w + j]; M[p * w + j] = t;
            }
        long double piv = M[k * w + k];
        for (int64_t j = 0; j < w; ++j) M[k * w + j] /= piv;
        for (int64_t i = 0; i < n; ++i) {
            if (i == k) continue;
            long double f = M[i * w + k];
            if (f == 0.0L) continue;
            for (int64_t j = 0; j < w; ++j) M[i * w + j] -= f * M[k * w + j];
        }
    }
    long double q = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
        long double row = 0.0L;
        for (int64_t j = 0; j < n; ++j) row += M[i * w + n + j] * (long double)z[j];
        q += (long double)z[i] * row;
    }
    *quad = q;
    free(M);
    return 0;
}
