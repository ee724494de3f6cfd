// FP64 tile Cholesky (Algorithm 2, dpotrf) by the right-looking tile algorithm
// of Section 5.2: for k = 0..T-1
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
#include "blocks.cuh"

namespace egs {

// ---- kernels --------------------------------------------------------------

// POTRF of the 64 x 64 sub-block at offset p of diagonal tile k; also zeroes
// rows p..p+63 to the right of the sub-block, so that once every sub-panel is
// done the tile holds L exactly (zero strict upper triangle).
__global__ void __launch_bounds__(256) k_potrf_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    double *A = tl.t64(k, k) + (size_t)p * b + p;
    if (!potrf64_smem(A, b, (int64_t)k * b + p, st)) return;
    for (int e = threadIdx.x; e < kIB * (b - p - kIB); e += 256) {
        const int r = e / (b - p - kIB), c = e % (b - p - kIB);
        A[(size_t)r * b + kIB + c] = 0.0;
    }
}

// Inside diagonal tile k: rows p + 64 + 16 * blockIdx.x solve against the
// factored 64 x 64 sub-block at p (16 rows per CTA: more SMs on the chain).
__global__ void __launch_bounds__(256) k_trsm_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    double *A = tl.t64(k, k);
    const int r0 = p + kIB + 16 * (int)blockIdx.x;
    trsm_rows<16>(A + (size_t)p * b + p, b, A + (size_t)r0 * b + p, b, kIB);
}

// Inside diagonal tile k: rank-64 update of the trailing lower part after
// sub-panel p, in 32 x 32 blocks (bi >= bj).
__global__ void __launch_bounds__(256) k_syrk_sub(Tiles tl, int k, int p, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    double *A = tl.t64(k, k);
    int bi, bj;
    tri_decode((int64_t)blockIdx.x, bi, bj);
    const int q = p + kIB;
    const int ri = q + 32 * bi, rj = q + 32 * bj;
    gemm_sub32(A + (size_t)ri * b + p, b, A + (size_t)rj * b + p, b, kIB, A + (size_t)ri * b + rj, b);
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
        const int nrest = (b - p - kIB) / 16;   // 16-row TRSM blocks
        const int n32 = (b - p - kIB) / 32;     // 32 x 32 SYRK blocks per side
        if (nrest > 0) {
            EGS_LAUNCH(kt, KC_POTRF, s, k_trsm_sub<<<(unsigned)nrest, 256, 0, s>>>(tl, k, p, st));
            EGS_LAUNCH(kt, KC_POTRF, s, k_syrk_sub<<<(unsigned)(n32 * (n32 + 1) / 2), 256, 0, s>>>(tl, k, p, st));
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

// The same update in 32 x 32 sub-blocks, for launches too small to fill the
// GPU with 64 x 64 blocks.
__global__ void __launch_bounds__(256) k_update_f64_32(Tiles tl, int k, DevStatus *st)
{
    if (failed(st)) return;
    const int b = tl.b;
    int mm, nn;
    tri_decode((int64_t)blockIdx.x, mm, nn);
    const int m = k + 1 + mm, nc = k + 1 + nn;
    const int nsub = b >> 5;
    const int sr = (int)blockIdx.y / nsub, sc = (int)blockIdx.y % nsub;
    if (m == nc && sc > sr) return;
    gemm_sub32(tl.t64(m, k) + (size_t)sr * 32 * b, b, tl.t64(nc, k) + (size_t)sc * 32 * b, b, b,
               tl.t64(m, nc) + (size_t)sr * 32 * b + sc * 32, b);
}

cudaError_t launch_update_f64(const Tiles &tl, int k, int64_t ntri, DevStatus *st, cudaStream_t s, KernelTimer *kt,
                              int cls)
{
    if (ntri <= 0) return cudaSuccess;
    const int nsub = tl.b / 64;
    if (ntri * nsub * (nsub + 1) / 2 < 304) {
        const int n32 = tl.b / 32;
        EGS_LAUNCH(kt, cls, s, k_update_f64_32<<<dim3((unsigned)ntri, (unsigned)(n32 * n32)), 256, 0, s>>>(tl, k, st));
    } else {
        EGS_LAUNCH(kt, cls, s, k_update_f64<<<dim3((unsigned)ntri, (unsigned)(nsub * nsub)), 256, 0, s>>>(tl, k, st));
    }
    return cudaGetLastError();
}

cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const int T = g.T;
    const Tiles tl{tiles, nullptr, g.b, T, T};
    for (int k = 0; k < T; ++k) {
        if (kt) kt->step = k;
        cudaError_t e = launch_potrf_diag(tl, k, st, s, kt);
        if (e != cudaSuccess) return e;
        if (k + 1 < T) {
            e = launch_trsm_f64(tl, k, T - k - 1, st, s, kt);
            if (e != cudaSuccess) return e;
            e = launch_update_f64(tl, k, (int64_t)(T - k - 1) * (T - k) / 2, st, s, kt);
            if (e != cudaSuccess) return e;
        }
    }
    if (kt) kt->step = -1;
    return cudaGetLastError();
}

}  // namespace egs
