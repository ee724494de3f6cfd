// Forward solve L y = Z on the lower-tile layout (Algorithm 2, dtrsm; the
// text of Section 6.5 writes it as L Z_new = Z_old), fused with the
// log-determinant log|Sigma| = 2 sum_i log L_ii (Section 6.1, taken in log
// form) and the dot product y^T y (Algorithm 2, computeDotProduct), then the
// assembly l = -1/2 y^T y - 1/2 log|Sigma| - n/2 log(2 pi) (Eq. 1).
//
// Column-oriented block substitution: for k = 0..T-1, the diagonal kernel
// solves tile k in place and records its two partial sums; the panel kernel
// then subtracts L_mk y_k from every later block (one CTA owns each output
// row, so the update order is fixed).  The whole solve reads each stored
// tile of L exactly once.  Reductions are fixed-order trees, so results are
// bitwise reproducible.
#include "blocks.cuh"

namespace egs {

__device__ __forceinline__ bool failed_s(const DevStatus *st)
{
    return *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

__global__ void k_pad_vector(const double *__restrict__ z, int64_t n, double *__restrict__ zpad, int64_t npad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npad) zpad[i] = (i < n) ? z[i] : 0.0;
}

// Diagonal block: y_k = L_kk^-1 r_k in place, blockDim.x = b threads.
__global__ void __launch_bounds__(1024) k_trsv_diag_f64(Tiles tl, int k, double *__restrict__ zpad,
                                                        double *__restrict__ partials, DevStatus *st)
{
    if (failed_s(st)) return;
    __shared__ double ldq[2];
    trsv_fwd_tile(tl.t64(k, k), tl.b, zpad + (size_t)k * tl.b, partials ? ldq : nullptr);
    if (partials && threadIdx.x == 0) {
        partials[k] = ldq[0];
        partials[tl.T + k] = ldq[1];
    }
}

// Panel: z_m -= L_mk y_k for m = k+1..T-1.  grid = (T-k-1, b/64), 256
// threads; each warp owns 8 rows and reduces each row's dot product with a
// fixed shuffle tree.  Tiles may be FP64 or (mixed mode) FP32.
__global__ void __launch_bounds__(256) k_gemv_panel(Tiles tl, int k, const double *ysrc, double *zpad,
                                                    const DevStatus *st)
{
    if (failed_s(st)) return;
    extern __shared__ double ys[];
    const int b = tl.b;
    const int m = k + 1 + (int)blockIdx.x;
    const int r0 = (int)blockIdx.y * 64;
    const bool f64 = tl.is64(m, k);
    float *ys32 = reinterpret_cast<float *>(ys + b);
    for (int c = threadIdx.x; c < b; c += 256) {
        const double v = ysrc[(size_t)k * b + c];
        ys[c] = v;
        ys32[c] = (float)v;
    }
    __syncthreads();
    if (f64) gemv_rows(tl.t64(m, k), b, r0, ys, zpad + (size_t)m * b);
    else gemv_rows_f32(tl.t32(m, k), b, r0, ys32, zpad + (size_t)m * b);
}

// l = -1/2 quad - 1/2 logdet - n/2 log(2 pi) from the per-tile partials.
__global__ void k_finalize(const double *__restrict__ partials, int T, int64_t n, DevStatus *st)
{
    __shared__ double red[256];
    double a = 0.0, q = 0.0;
    for (int t = threadIdx.x; t < T; t += 256) {
        a += partials[t];
        q += partials[T + t];
    }
    const double lsum = block_sum(a, red);
    __syncthreads();
    const double qsum = block_sum(q, red);
    if (threadIdx.x == 0) {
        if (failed_s(st)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            st->result[0] = st->result[1] = st->result[2] = nan;
        } else {
            const double logdet = 2.0 * lsum;
            st->result[0] = -0.5 * qsum - 0.5 * logdet - 0.5 * (double)n * 1.8378770664093454836;  // log(2 pi)
            st->result[1] = logdet;
            st->result[2] = qsum;
        }
    }
}

// Z = L e over the lower tiles of L (Algorithm 1, dtrmm): out[i*b + r] =
// sum_{j <= i} L_ij[r][:] . e_j, one warp per row, fixed shuffle tree.
// Diagonal tiles hold L with a zero strict upper triangle.  grid = (T, b/8).
__global__ void __launch_bounds__(256) k_trmv_lower(const double *__restrict__ tiles, int b, int T,
                                                    const double *__restrict__ e, double *__restrict__ out,
                                                    const DevStatus *st)
{
    if (failed_s(st)) return;
    const int i = (int)blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (int)blockIdx.y * 8 + warp;
    const size_t bb = (size_t)b * b;
    double s = 0.0;
    for (int j = 0; j <= i; ++j) {
        const double *row = tiles + (size_t)tile_linear(i, j) * bb + (size_t)r * b;
        const double *ej = e + (size_t)j * b;
        for (int c = lane; c < b; c += 32) s = fma(row[c], ej[c], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[(size_t)i * b + r] = s;
}

cudaError_t launch_trmv_lower(const double *tiles, const TileGeom &g, const double *epad, double *out,
                              const DevStatus *st, cudaStream_t s)
{
    k_trmv_lower<<<dim3((unsigned)g.T, (unsigned)(g.b / 8)), 256, 0, s>>>(tiles, g.b, g.T, epad, out, st);
    return cudaGetLastError();
}

cudaError_t launch_pad_vector(const double *z, int64_t n, double *zpad, int64_t npad, cudaStream_t s, KernelTimer *kt)
{
    const unsigned blocks = (unsigned)((npad + 255) / 256);
    EGS_LAUNCH(kt, KC_OTHER, s, k_pad_vector<<<blocks, 256, 0, s>>>(z, n, zpad, npad));
    return cudaGetLastError();
}

cudaError_t launch_forward_solve(const Tiles &tl, double *zpad, double *partials, DevStatus *st, cudaStream_t s,
                                 KernelTimer *kt)
{
    const int b = tl.b, T = tl.T;
    for (int k = 0; k < T; ++k) {
        EGS_LAUNCH(kt, KC_TRSV, s, k_trsv_diag_f64<<<1, b, 0, s>>>(tl, k, zpad, partials, st));
        if (k + 1 < T)
            EGS_LAUNCH(kt, KC_TRSV, s,
                       k_gemv_panel<<<dim3((unsigned)(T - k - 1), (unsigned)(b / 64)), 256,
                                      (size_t)b * (sizeof(double) + sizeof(float)), s>>>(tl, k, zpad, zpad, st));
    }
    return cudaGetLastError();
}

cudaError_t launch_gemv_panel(const Tiles &tl, int k, const double *ysrc, double *zpad, const DevStatus *st,
                              cudaStream_t s, KernelTimer *kt)
{
    if (k + 1 >= tl.T) return cudaSuccess;
    EGS_LAUNCH(kt, KC_TRSV, s,
               k_gemv_panel<<<dim3((unsigned)(tl.T - k - 1), (unsigned)(tl.b / 64)), 256,
                              (size_t)tl.b * (sizeof(double) + sizeof(float)), s>>>(tl, k, ysrc, zpad, st));
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int T, int64_t n, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    EGS_LAUNCH(kt, KC_OTHER, s, k_finalize<<<1, 256, 0, s>>>(partials, T, n, st));
    return cudaGetLastError();
}

cudaError_t launch_trsv_tiles_f64(const double *tiles, const TileGeom &g, double *zpad, double *partials,
                                  DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const Tiles tl{const_cast<double *>(tiles), nullptr, g.b, g.T, g.T};
    cudaError_t e = launch_forward_solve(tl, zpad, partials, st, s, kt);
    if (e != cudaSuccess) return e;
    return launch_finalize(partials, g.T, g.n, st, s, kt);
}

}  // namespace egs
