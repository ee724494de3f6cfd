// Kriging prediction (Section 2.3, Eq. 5; Algorithm 3): with zero means,
//   Z_1 = Sigma_12 Sigma_22^-1 Z_2,
// Sigma_22 (n x n) the covariance of the observed locations and Sigma_12
// (m x n) the cross-covariance of the new locations with them.  Algorithm 3
// solves Sigma_22 X = Z_2 (dposv) and multiplies by Sigma_12 (dgemm).  Here
// the solve reuses one likelihood evaluation's factorisation (FP64: POTRF
// and the forward solve, then the backward solve; mixed precision: the
// refined x = Sigma^-1 Z of the evaluation), and Sigma_12 is never stored:
// one kernel forms each cross-covariance entry from the coordinates in
// registers and accumulates it against X (generation fused into the dgemm,
// which is a matrix-vector product for one measurement vector).
#include "egs_internal.cuh"
#include "matern.cuh"

namespace egs {

namespace {

constexpr int PB = 32;       // new locations per CTA
constexpr int GROUP = 8;     // threads per new location
constexpr int OCHUNK = 256;  // observed locations staged per pass

// z_new[i] = sum_j C(||s_i - s_j||) x_j for the PB new locations of this CTA.
// Thread t handles new location t / GROUP and observed locations
// t % GROUP + GROUP q of every staged chunk; the GROUP partial sums of a
// location are combined by a fixed shuffle tree, so results are bitwise
// reproducible.
__global__ void __launch_bounds__(256) k_predict(const double *__restrict__ Xn, const double *__restrict__ Yn,
                                                 int64_t m, const double *__restrict__ Xo,
                                                 const double *__restrict__ Yo, const double *__restrict__ x,
                                                 int64_t n, const __grid_constant__ egs_matern_params Pg,
                                                 double *__restrict__ z_new, const DevStatus *st)
{
    if (*(volatile const unsigned long long *)&st->fail_index != kNoFail) return;
    __shared__ egs_matern_params Ps;
    __shared__ double sx[OCHUNK], sy[OCHUNK], sv[OCHUNK];
    {
        const double *s = reinterpret_cast<const double *>(&Pg);
        double *d = reinterpret_cast<double *>(&Ps);
        for (int i = threadIdx.x; i < (int)(sizeof(egs_matern_params) / sizeof(double)); i += blockDim.x) d[i] = s[i];
    }
    const int li = threadIdx.x / GROUP, g = threadIdx.x % GROUP;
    const int64_t i = (int64_t)blockIdx.x * PB + li;
    const double xi = i < m ? Xn[i] : 0.0, yi = i < m ? Yn[i] : 0.0;
    const double inv_th2 = Pg.inv_th2;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += OCHUNK) {
        __syncthreads();
        for (int t = threadIdx.x; t < OCHUNK; t += blockDim.x) {
            const int64_t j = j0 + t;
            sx[t] = j < n ? Xo[j] : 0.0;
            sy[t] = j < n ? Yo[j] : 0.0;
            sv[t] = j < n ? x[j] : 0.0;
        }
        __syncthreads();
        const int cnt = (n - j0 < OCHUNK) ? (int)(n - j0) : OCHUNK;
        for (int t = g; t < cnt; t += GROUP) {
            acc = fma(matern_eval(&Ps, loc_dist(&Ps, xi, yi, sx[t], sy[t]) * inv_th2), sv[t], acc);
        }
    }
#pragma unroll
    for (int off = GROUP / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (g == 0 && i < m) z_new[i] = acc;
}

}  // namespace

}  // namespace egs

using namespace egs;

extern "C" egs_status egs_predict(const double *locs_obs, const double *z_obs, int64_t n, const double *locs_new,
                                  int64_t m, const double theta[3], egs_precision p, const egs_opts *opts,
                                  double *z_new, egs_info *info, void *stream)
{
    if (!locs_obs || !z_obs || !locs_new || !z_new) return set_error(EGS_ERR_ARG, "egs_predict: NULL pointer");
    if (m < 1) return set_error(EGS_ERR_ARG, "egs_predict: m = %lld must be >= 1", (long long)m);
    EvalSetup es;
    egs_status sc = eval_setup(n, theta, p, opts, &es);
    if (sc != EGS_OK) return sc;
    cudaStream_t s = (cudaStream_t)stream;
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t extra_new = a256((size_t)2 * m * sizeof(double)), extra_out = a256((size_t)m * sizeof(double));
    char *ws = nullptr;
    const Allocator A = current_allocator();
    const size_t wbytes = es.need + extra_new + extra_out;
    cudaError_t e = dev_alloc(A, (void **)&ws, wbytes, s);
    if (e != cudaSuccess) return cuda_error(e, "egs_predict workspace");
    const double *dlocs = locs_obs, *dz = z_obs, *dnew = locs_new;
    double *dout = z_new;
    if (!is_device_ptr(locs_obs)) {
        dlocs = (const double *)(ws + es.locs_off);
        e = cudaMemcpyAsync((void *)dlocs, locs_obs, (size_t)2 * n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && !is_device_ptr(z_obs)) {
        dz = (const double *)(ws + es.z_off);
        e = cudaMemcpyAsync((void *)dz, z_obs, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && !is_device_ptr(locs_new)) {
        dnew = (const double *)(ws + es.need);
        e = cudaMemcpyAsync((void *)dnew, locs_new, (size_t)2 * m * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    const bool host_out = !is_device_ptr(z_new);
    if (host_out) dout = (double *)(ws + es.need + extra_new);
    KernelTimer kt;
    // Algorithm 3, the solve: Sigma_22, its factorisation and X = Sigma_22^-1 Z_2
    if (e == cudaSuccess) e = eval_enqueue(es, dlocs, dz, ws, s, &kt, nullptr);
    if (e == cudaSuccess) e = finish_solution(es, ws, s);
    // Algorithm 3, the product: Z_1 = Sigma_12 X, Sigma_12 formed on the fly
    if (e == cudaSuccess) {
        k_predict<<<(unsigned)((m + PB - 1) / PB), 256, 0, s>>>(dnew, dnew + m, m, dlocs, dlocs + n,
                                                               eval_solution(es, ws), n, es.P, dout,
                                                               eval_status(es, ws));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && host_out) e = cudaMemcpyAsync(z_new, dout, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s);
    DevStatus h;
    int herr = 0;
    if (e == cudaSuccess && es.mixed) e = cudaMemcpyAsync(&herr, ws + es.ML.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, eval_status(es, ws), sizeof(h), cudaMemcpyDeviceToHost, s);
    dev_free(A, ws, wbytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "egs_predict");
    if (herr || h.timeout) return set_error(EGS_ERR_TIMEOUT, "egs_predict: a bounded device wait timed out");
    if (info) {
        fill_info(es, h, info);
        info->launches = kt.launches + 1;
    }
    if (h.fail_index != kNoFail)
        return set_error(EGS_ERR_NOT_PD, "egs_predict: Sigma_22 not positive definite at row %lld",
                         (long long)h.fail_index);
    if (!mixed_result_ok(es, h))
        return set_error(EGS_ERR_INACCURATE, "egs_predict: the mixed factor is too inexact for Sigma_22; use EGS_FP64");
    return EGS_OK;
}
