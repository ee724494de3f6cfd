// FP64 tile Cholesky (Algorithm 2, dpotrf) on the lower-tile layout, by the
// right-looking tile algorithm of Section 4.2: for k = 0..T-1
//   POTRF  L_kk = chol(A_kk)
//   TRSM   A_mk <- A_mk L_kk^-T            (m > k)
//   SYRK   A_mm <- A_mm - A_mk A_mk^T       (m > k)
//   GEMM   A_mn <- A_mn - A_mk A_nk^T       (m > n > k)
// SYRK and GEMM share one kernel (a diagonal output tile skips its upper
// sub-blocks).
//
// GB300's FP64 rate is 2 DFMA per clock per SM (about 1.2 TFLOP/s for the
// chip), so these kernels are FP64-pipe bound whatever their memory traffic:
// the design goal is to keep every SM's FP64 pipe busy, not to save bytes.
// Every output element is updated by exactly one thread in a fixed order, so
// results are bitwise reproducible.
#include "egs_internal.cuh"

namespace egs {

constexpr int kPW = 16;  // POTRF panel width

__device__ __forceinline__ bool failed(const DevStatus *st)
{
    return *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

__device__ __forceinline__ void tile_decode2(int64_t t, int &i, int &j)
{
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    i = ii;
    j = (int)(t - (int64_t)ii * (ii + 1) / 2);
}

// ---------------------------------------------------------------------------
// POTRF of diagonal tile k, one CTA of 256 threads, right-looking over
// 16-column panels: (1) one warp factors the 16 x 16 diagonal block in shared
// memory; (2) the rows below solve against it; (3) rank-16 update of the
// trailing lower triangle.  Dynamic shared memory: b x 17 doubles.
// A pivot that is not positive records its global row in st->fail_index.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_potrf_diag_f64(double *tiles, int b, int k, DevStatus *st)
{
    if (failed(st)) return;
    extern __shared__ double pan[];  // [b][kPW + 1]
    __shared__ double dblk[kPW][kPW + 1];
    __shared__ int fail_j;
    double *A = tiles + (size_t)tile_linear(k, k) * (size_t)b * (size_t)b;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) fail_j = -1;
    __syncthreads();
    for (int p0 = 0; p0 < b; p0 += kPW) {
        for (int e = tid; e < kPW * kPW; e += 256) {
            const int i = e / kPW, j = e % kPW;
            if (j <= i) dblk[i][j] = A[(size_t)(p0 + i) * b + p0 + j];
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
            if (tid == 0) atomicMin(&st->fail_index, (unsigned long long)((int64_t)k * b + fail_j));
            return;
        }
        // write back the factored diagonal block
        for (int e = tid; e < kPW * kPW; e += 256) {
            const int i = e / kPW, j = e % kPW;
            if (j <= i) A[(size_t)(p0 + i) * b + p0 + j] = dblk[i][j];
        }
        // (2) rows below the block: x L_blk^T = a
        for (int i = p0 + kPW + tid; i < b; i += 256) {
            double x[kPW];
            double *row = A + (size_t)i * b + p0;
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
        // (3) trailing update of the lower triangle, rows/cols >= p0 + kPW
        const int q0 = p0 + kPW;
        for (int i = q0 + warp; i < b; i += 8) {
            double li[kPW];
#pragma unroll
            for (int l = 0; l < kPW; ++l) li[l] = pan[(size_t)i * (kPW + 1) + l];
            double *row = A + (size_t)i * b;
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
    // zero the strict upper triangle so the tile holds L exactly
    for (int i = warp; i < b; i += 8)
        for (int j = i + 1 + lane; j < b; j += 32) A[(size_t)i * b + j] = 0.0;
}

// ---------------------------------------------------------------------------
// TRSM on the panel below tile k: X L_kk^T = A_mk for m = k+1..T-1.  One CTA
// solves 64 rows of one tile, sweeping 32-column blocks: a GEMM-style update
// with the already-solved columns, then a 32-wide substitution in shared
// memory.  grid = (T - k - 1, b / 64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_trsm_panel_f64(double *tiles, int b, int k, DevStatus *st)
{
    if (failed(st)) return;
    const int m = k + 1 + (int)blockIdx.x;
    const int r0 = (int)blockIdx.y * 64;
    const size_t bb = (size_t)b * (size_t)b;
    const double *L = tiles + (size_t)tile_linear(k, k) * bb;
    double *A = tiles + (size_t)tile_linear(m, k) * bb + (size_t)r0 * b;
    __shared__ double Xs[64][kPW + 1];
    __shared__ double Ls[32][kPW + 1];
    __shared__ double Ab[64][33];
    __shared__ double Ld[32][33];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    for (int c0 = 0; c0 < b; c0 += 32) {
        double acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = A[(size_t)(ty * 8 + i) * b + c0 + tx];
        for (int p = 0; p < c0; p += kPW) {
            for (int e = tid; e < 64 * kPW; e += 256) {
                const int r = e >> 4, l = e & 15;
                Xs[r][l] = A[(size_t)r * b + p + l];
            }
            for (int e = tid; e < 32 * kPW; e += 256) {
                const int c = e >> 4, l = e & 15;
                Ls[c][l] = L[(size_t)(c0 + c) * b + p + l];
            }
            __syncthreads();
#pragma unroll
            for (int l = 0; l < kPW; ++l) {
                const double lv = Ls[tx][l];
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fma(-Xs[ty * 8 + i][l], lv, acc[i]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) Ab[ty * 8 + i][tx] = acc[i];
        for (int e = tid; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            Ld[r][c] = (c <= r) ? L[(size_t)(c0 + r) * b + c0 + c] : 0.0;
        }
        __syncthreads();
        if (tid < 64) {
            for (int j = 0; j < 32; ++j) {
                double s = Ab[tid][j];
                for (int l = 0; l < j; ++l) s -= Ab[tid][l] * Ld[j][l];
                Ab[tid][j] = s / Ld[j][j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) A[(size_t)(ty * 8 + i) * b + c0 + tx] = Ab[ty * 8 + i][tx];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Trailing update at step k: C_mn -= A_mk A_nk^T for T > m >= n > k.
// One CTA computes a 64 x 64 sub-block with 4 x 4 outputs per thread (rows
// ty + 16 i, columns tx + 16 j, so global accesses of a half-warp are 128
// contiguous bytes).  grid = ((T-k-1)(T-k)/2, (b/64)^2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update_f64(double *tiles, int b, int k, DevStatus *st)
{
    if (failed(st)) return;
    int mm, nn;
    tile_decode2((int64_t)blockIdx.x, mm, nn);
    const int m = k + 1 + mm, nc = k + 1 + nn;
    const int nsub = b >> 6;
    const int sr = (int)blockIdx.y / nsub, sc = (int)blockIdx.y % nsub;
    if (m == nc && sc > sr) return;
    const size_t bb = (size_t)b * (size_t)b;
    const double *Am = tiles + (size_t)tile_linear(m, k) * bb + (size_t)sr * 64 * b;
    const double *An = tiles + (size_t)tile_linear(nc, k) * bb + (size_t)sc * 64 * b;
    double *C = tiles + (size_t)tile_linear(m, nc) * bb + (size_t)sr * 64 * b + sc * 64;
    __shared__ double As[kPW][65];
    __shared__ double Bs[kPW][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int p = 0; p < b; p += kPW) {
        for (int e = tid; e < 64 * kPW; e += 256) {
            const int r = e >> 4, l = e & 15;
            As[l][r] = Am[(size_t)r * b + p + l];
            Bs[l][r] = An[(size_t)r * b + p + l];
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
        for (int j = 0; j < 4; ++j) C[(size_t)(ty + 16 * i) * b + tx + 16 * j] -= acc[i][j];
}

cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const int b = g.b, T = g.T, nsub = b / 64;
    const size_t smem = (size_t)b * (kPW + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_potrf_diag_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < T; ++k) {
        EGS_LAUNCH(kt, KC_POTRF, s, k_potrf_diag_f64<<<1, 256, smem, s>>>(tiles, b, k, st));
        if (k + 1 < T) {
            EGS_LAUNCH(kt, KC_TRSM, s,
                       k_trsm_panel_f64<<<dim3((unsigned)(T - k - 1), (unsigned)nsub), 256, 0, s>>>(tiles, b, k, st));
            const int64_t nt = (int64_t)(T - k - 1) * (T - k) / 2;
            EGS_LAUNCH(kt, KC_UPDATE, s,
                       k_update_f64<<<dim3((unsigned)nt, (unsigned)(nsub * nsub)), 256, 0, s>>>(tiles, b, k, st));
        }
    }
    return cudaGetLastError();
}

}  // namespace egs
