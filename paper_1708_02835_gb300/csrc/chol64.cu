// FP64 tile Cholesky (Algorithm 2, dpotrf) by the right-looking tile algorithm
// of Section 4.2: for k = 0..T-1
//   POTRF  L_kk = chol(A_kk)
//   TRSM   A_mk <- A_mk L_kk^-T            (m > k)
//   SYRK   A_mm <- A_mm - A_mk A_mk^T       (m > k)
//   GEMM   A_mn <- A_mn - A_mk A_nk^T       (m > n > k)
// SYRK and GEMM share one kernel (a diagonal output tile skips its upper
// sub-blocks).
//
// The diagonal POTRF is itself blocked: 64-wide sub-panels, each factored by
// one CTA, with the rows below solved and the trailing part of the tile
// updated by many CTAs, so that the factorisation's critical path uses many
// SMs instead of one.
//
// GB300's FP64 rate is 2 DFMA per clock per SM (about 1.2 TFLOP/s for the
// chip), so these kernels are FP64-pipe bound whatever their memory traffic:
// the design goal is to keep every SM's FP64 pipe busy, not to save bytes.
// Every output element is updated by exactly one thread in a fixed order, so
// results are bitwise reproducible.
#include "egs_internal.cuh"

namespace egs {

constexpr int kPW = 16;  // panel width inside the single-CTA POTRF
constexpr int kIB = 64;  // sub-panel width of the blocked diagonal POTRF

__device__ __forceinline__ bool failed(const DevStatus *st)
{
    return *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

__device__ __forceinline__ void tri_decode(int64_t t, int &i, int &j)
{
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    i = ii;
    j = (int)(t - (int64_t)ii * (ii + 1) / 2);
}

// ---------------------------------------------------------------------------
// Cholesky of an nb x nb block at A (row stride ld) by one CTA of 256 threads,
// right-looking over 16-column panels: one warp factors the 16 x 16 diagonal
// block in shared memory, the rows below solve against it, then a rank-16
// update of the trailing lower triangle.  pan: nb x 17 doubles of shared
// memory.  A pivot that is not positive records row0 + its row in
// st->fail_index and returns false.  The strict upper triangle is zeroed.
// ---------------------------------------------------------------------------
__device__ bool potrf_block(double *A, int nb, int ld, int64_t row0, DevStatus *st, double *pan)
{
    __shared__ double dblk[kPW][kPW + 1];
    __shared__ int fail_j;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) fail_j = -1;
    __syncthreads();
    for (int p0 = 0; p0 < nb; p0 += kPW) {
        for (int e = tid; e < kPW * kPW; e += 256) {
            const int i = e / kPW, j = e % kPW;
            if (j <= i) dblk[i][j] = A[(size_t)(p0 + i) * ld + p0 + j];
        }
        __syncthreads();
        if (warp == 0) {
            for (int j = 0; j < kPW; ++j) {
                if (lane == 0) {
                    const double d = dblk[j][j];
                    if (!(d > 0.0)) fail_j = p0 + j;
                    else dblk[j][j] = sqrt(d);
                }
                __syncwarp();
                if (fail_j >= 0) break;
                const double ljj = dblk[j][j];
                if (lane > j && lane < kPW) dblk[lane][j] /= ljj;
                __syncwarp();
                if (lane > j && lane < kPW) {
                    const double lij = dblk[lane][j];
                    for (int l = j + 1; l <= lane; ++l) dblk[lane][l] -= lij * dblk[l][j];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (fail_j >= 0) {
            if (tid == 0) atomicMin(&st->fail_index, (unsigned long long)(row0 + fail_j));
            return false;
        }
        for (int e = tid; e < kPW * kPW; e += 256) {
            const int i = e / kPW, j = e % kPW;
            if (j <= i) A[(size_t)(p0 + i) * ld + p0 + j] = dblk[i][j];
        }
        for (int i = p0 + kPW + tid; i < nb; i += 256) {
            double x[kPW];
            double *row = A + (size_t)i * ld + p0;
#pragma unroll
            for (int j = 0; j < kPW; ++j) x[j] = row[j];
#pragma unroll
            for (int j = 0; j < kPW; ++j) {
                double s = x[j];
#pragma unroll
                for (int l = 0; l < j; ++l) s -= x[l] * dblk[j][l];
                x[j] = s / dblk[j][j];
            }
#pragma unroll
            for (int j = 0; j < kPW; ++j) {
                row[j] = x[j];
                pan[(size_t)i * (kPW + 1) + j] = x[j];
            }
        }
        __syncthreads();
        const int q0 = p0 + kPW;
        for (int i = q0 + warp; i < nb; i += 8) {
            double li[kPW];
#pragma unroll
            for (int l = 0; l < kPW; ++l) li[l] = pan[(size_t)i * (kPW + 1) + l];
            double *row = A + (size_t)i * ld;
            for (int j = q0 + lane; j <= i; j += 32) {
                const double *lj = pan + (size_t)j * (kPW + 1);
                double acc = 0.0;
#pragma unroll
                for (int l = 0; l < kPW; ++l) acc = fma(li[l], lj[l], acc);
                row[j] -= acc;
            }
        }
        __syncthreads();
    }
    for (int i = warp; i < nb; i += 8)
        for (int j = i + 1 + lane; j < nb; j += 32) A[(size_t)i * ld + j] = 0.0;
    return true;
}

// ---------------------------------------------------------------------------
// X L^T = A for RB rows (RB in {8, 16, 64}): X and A at Xp (row stride ldx,
// ncols columns), L lower ncols x ncols at Lp (row stride ldl).  32-column
// blocks: a GEMM-style update with the already-solved columns, then a
// 32-wide substitution in shared memory.  256 threads; fewer rows per CTA put
// more SMs on a panel when the panel is short.
// ---------------------------------------------------------------------------
template <int RB>
__device__ void trsm_rows(const double *Lp, int ldl, double *Xp, int ldx, int ncols)
{
    constexpr int RPG = RB / 8;  // rows per thread group (8 groups of 32 threads)
    __shared__ double Xs[RB][kPW + 1];
    __shared__ double Ls[32][kPW + 1];
    __shared__ double Ab[RB][33];
    __shared__ double Ld[32][33];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    for (int c0 = 0; c0 < ncols; c0 += 32) {
        double acc[RPG];
#pragma unroll
        for (int i = 0; i < RPG; ++i) acc[i] = Xp[(size_t)(ty * RPG + i) * ldx + c0 + tx];
        for (int p = 0; p < c0; p += kPW) {
            for (int e = tid; e < RB * kPW; e += 256) {
                const int r = e >> 4, l = e & 15;
                Xs[r][l] = Xp[(size_t)r * ldx + p + l];
            }
            for (int e = tid; e < 32 * kPW; e += 256) {
                const int c = e >> 4, l = e & 15;
                Ls[c][l] = Lp[(size_t)(c0 + c) * ldl + p + l];
            }
            __syncthreads();
#pragma unroll
            for (int l = 0; l < kPW; ++l) {
                const double lv = Ls[tx][l];
#pragma unroll
                for (int i = 0; i < RPG; ++i) acc[i] = fma(-Xs[ty * RPG + i][l], lv, acc[i]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < RPG; ++i) Ab[ty * RPG + i][tx] = acc[i];
        for (int e = tid; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            Ld[r][c] = (c <= r) ? Lp[(size_t)(c0 + r) * ldl + c0 + c] : 0.0;
        }
        __syncthreads();
        if (tid < RB) {
            for (int j = 0; j < 32; ++j) {
                double s = Ab[tid][j];
                for (int l = 0; l < j; ++l) s -= Ab[tid][l] * Ld[j][l];
                Ab[tid][j] = s / Ld[j][j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RPG; ++i) Xp[(size_t)(ty * RPG + i) * ldx + c0 + tx] = Ab[ty * RPG + i][tx];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// C (64 x 64, row stride ldc) -= Am (64 x K) An (64 x K)^T with row strides
// lda, ldb.  4 x 4 outputs per thread (rows ty + 16 i, columns tx + 16 j, so a
// half-warp touches 128 contiguous bytes).  256 threads.
// ---------------------------------------------------------------------------
__device__ void gemm_sub64(const double *Am, int lda, const double *An, int ldb, int K, double *C, int ldc)
{
    __shared__ double As[kPW][65];
    __shared__ double Bs[kPW][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int p = 0; p < K; p += kPW) {
        for (int e = tid; e < 64 * kPW; e += 256) {
            const int r = e >> 4, l = e & 15;
            As[l][r] = Am[(size_t)r * lda + p + l];
            Bs[l][r] = An[(size_t)r * ldb + p + l];
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < kPW; ++l) {
            double a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[l][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[l][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) C[(size_t)(ty + 16 * i) * ldc + tx + 16 * j] -= acc[i][j];
}

// ---- kernels --------------------------------------------------------------

// POTRF of the 64 x 64 sub-block at offset p of diagonal tile k; also zeroes
// rows p..p+63 to the right of the sub-block, so that once every sub-panel is
// done the tile holds L exactly (zero strict upper triangle).
__global__ void __launch_bounds__(256) k_potrf_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    __shared__ double pan[kIB * (kPW + 1)];
    const int b = tl.b;
    double *A = tl.t64(k, k) + (size_t)p * b + p;
    if (!potrf_block(A, kIB, b, (int64_t)k * b + p, st, pan)) return;
    for (int e = threadIdx.x; e < kIB * (b - p - kIB); e += 256) {
        const int r = e / (b - p - kIB), c = e % (b - p - kIB);
        A[(size_t)r * b + kIB + c] = 0.0;
    }
}

// Inside diagonal tile k: rows p + 64 + 64 * blockIdx.x solve against the
// factored 64 x 64 sub-block at p.
__global__ void __launch_bounds__(256) k_trsm_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    double *A = tl.t64(k, k);
    const int r0 = p + kIB + 64 * (int)blockIdx.x;
    trsm_rows<64>(A + (size_t)p * b + p, b, A + (size_t)r0 * b + p, b, kIB);
}

// Inside diagonal tile k: rank-64 update of the trailing lower part after
// sub-panel p, in 64 x 64 blocks (bi >= bj).
__global__ void __launch_bounds__(256) k_syrk_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    double *A = tl.t64(k, k);
    int bi, bj;
    tri_decode((int64_t)blockIdx.x, bi, bj);
    const int q = p + kIB;
    const int ri = q + 64 * bi, rj = q + 64 * bj;
    gemm_sub64(A + (size_t)ri * b + p, b, A + (size_t)rj * b + p, b, kIB, A + (size_t)ri * b + rj, b);
}

// TRSM on the panel below tile k: rows m = k+1+blockIdx.x, RB rows per CTA.
template <int RB>
__global__ void __launch_bounds__(256) k_trsm_panel_f64(Tiles tl, int k, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    const int m = k + 1 + (int)blockIdx.x;
    const int r0 = (int)blockIdx.y * RB;
    trsm_rows<RB>(tl.t64(k, k), b, tl.t64(m, k) + (size_t)r0 * b, b, b);
}

// Trailing update at step k for the first gridDim.x tiles of the trailing
// triangle (enumerated row by row: (k+1,k+1), (k+2,k+1), (k+2,k+2), ...):
// C_mn -= A_mk A_nk^T in 64 x 64 sub-blocks.  grid = (tiles, (b/64)^2).
__global__ void __launch_bounds__(256) k_update_f64(Tiles tl, int k, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    int mm, nn;
    tri_decode((int64_t)blockIdx.x, mm, nn);
    const int m = k + 1 + mm, nc = k + 1 + nn;
    const int nsub = b >> 6;
    const int sr = (int)blockIdx.y / nsub, sc = (int)blockIdx.y % nsub;
    if (m == nc && sc > sr) return;
    gemm_sub64(tl.t64(m, k) + (size_t)sr * 64 * b, b, tl.t64(nc, k) + (size_t)sc * 64 * b, b, b,
               tl.t64(m, nc) + (size_t)sr * 64 * b + sc * 64, b);
}

cudaError_t launch_potrf_diag(const Tiles &tl, int k, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const int b = tl.b;
    for (int p = 0; p < b; p += kIB) {
        EGS_LAUNCH(kt, KC_POTRF, s, k_potrf_sub<<<1, 256, 0, s>>>(tl, k, p, st));
        const int nrest = (b - p - kIB) / 64;
        if (nrest > 0) {
            EGS_LAUNCH(kt, KC_POTRF, s, k_trsm_sub<<<(unsigned)nrest, 256, 0, s>>>(tl, k, p, st));
            EGS_LAUNCH(kt, KC_POTRF, s, k_syrk_sub<<<(unsigned)(nrest * (nrest + 1) / 2), 256, 0, s>>>(tl, k, p, st));
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_trsm_f64(const Tiles &tl, int k, int nrows, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    if (nrows <= 0) return cudaSuccess;
    // enough 64-row CTAs to cover the SMs?  otherwise split rows finer
    if ((int64_t)nrows * (tl.b / 64) >= 304) {
        EGS_LAUNCH(kt, KC_TRSM, s,
                   k_trsm_panel_f64<64><<<dim3((unsigned)nrows, (unsigned)(tl.b / 64)), 256, 0, s>>>(tl, k, st));
    } else if ((int64_t)nrows * (tl.b / 16) >= 152) {
        EGS_LAUNCH(kt, KC_TRSM, s,
                   k_trsm_panel_f64<16><<<dim3((unsigned)nrows, (unsigned)(tl.b / 16)), 256, 0, s>>>(tl, k, st));
    } else {
        EGS_LAUNCH(kt, KC_TRSM, s,
                   k_trsm_panel_f64<8><<<dim3((unsigned)nrows, (unsigned)(tl.b / 8)), 256, 0, s>>>(tl, k, st));
    }
    return cudaGetLastError();
}

cudaError_t launch_update_f64(const Tiles &tl, int k, int64_t ntri, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    if (ntri <= 0) return cudaSuccess;
    const int nsub = tl.b / 64;
    EGS_LAUNCH(kt, KC_UPDATE, s, k_update_f64<<<dim3((unsigned)ntri, (unsigned)(nsub * nsub)), 256, 0, s>>>(tl, k, st));
    return cudaGetLastError();
}

cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const int T = g.T;
    const Tiles tl{tiles, nullptr, g.b, T, T};
    for (int k = 0; k < T; ++k) {
        cudaError_t e = launch_potrf_diag(tl, k, st, s, kt);
        if (e != cudaSuccess) return e;
        if (k + 1 < T) {
            e = launch_trsm_f64(tl, k, T - k - 1, st, s, kt);
            if (e != cudaSuccess) return e;
            e = launch_update_f64(tl, k, (int64_t)(T - k - 1) * (T - k) / 2, st, s, kt);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

}  // namespace egs
