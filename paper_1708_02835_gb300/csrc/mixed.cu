// Mixed-precision evaluation of Eq. 1 (Algorithm 2) with an FP64 diagonal band.
//
// Storage: tiles with i - j < band (the diagonal band) stay FP64; the others
// are FP32.  Per step k of the right-looking tile Cholesky (Section 5.2):
//   POTRF  L_kk in FP64;
//   TRSM   band rows (m - k < band) in FP64; the other rows in the FP32
//          mode as the product with W = L_kk^-1 (inverted in FP64) on tcgen05
//          in split TF32, in the TF32 / BF16 modes in FP32 arithmetic with
//          L_kk rounded to FP32; every solved tile is also written to the
//          panel buffer in the tensor-core operand format (TF32-rounded FP32,
//          split TF32 hi/lo pairs, or BF16);
//   UPDATE C_mn -= P_m P_n^T: when both P_m and P_n are FP64 band tiles the
//          update runs in FP64 (DFMA) on the unrounded values.  TF32 / BF16:
//          every other update runs on tcgen05 with FP32 accumulation
//          (tc_gemm.cu) and is subtracted in FP64 from band tiles and in FP32
//          from the others.  FP32 mode (split TF32): each update takes the
//          precision of its output tile, as in a mixed-precision tile
//          Cholesky that keeps the band in double -- band outputs in FP64 on
//          the stored FP32 / FP64 values (band x band on DFMA, the others as
//          exact BF16 slice products on tcgen05, ozaki.cu), off-band outputs
//          on tcgen05 as lo hi^T + hi lo^T + hi hi^T (FP32-accurate products).
// The log-determinant 2 sum log L_ii is reduced in FP64 from the FP64
// diagonal tiles.  The quadratic form Z^T Sigma^-1 Z is won back in FP64 by
// iterative refinement: x0 = L^-T L^-1 Z, r = Z - Sigma x0 with Sigma
// regenerated tile by tile (symv_regen.cu), x1 = x0 + L^-T L^-1 r, quad = Z^T x1.
#include "blocks.cuh"
#include "slices.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace egs {

namespace {

__device__ __forceinline__ bool mfailed(const DevStatus *st)
{
    return *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Element (row, col) of the panel operand buffer; row counts over all panel
// tiles ((T-1) b rows), col < b.  FMT 3 (split TF32) writes hi = tf32(v) and
// lo = tf32(v - hi) (v - hi is exact in FP32) as the row [hi | lo] of 2b
// floats; the update reads both halves of both operands and forms
// lo hi^T + hi lo^T + hi hi^T.
template <int FMT>
__device__ __forceinline__ void panel_store(void *panel, const Tiles &tl, size_t row, int col, float v)
{
    if (FMT == 3) {
        const size_t ld = 2 * (size_t)tl.b;
        float *pa = reinterpret_cast<float *>(panel) + row * ld + col;
        const float hi = to_tf32(v), lo = to_tf32(v - hi);
        pa[0] = hi;
        pa[tl.b] = lo;
    } else if (FMT == 2) {
        reinterpret_cast<float *>(panel)[row * tl.b + col] = to_tf32(v);
    } else {
        reinterpret_cast<__nv_bfloat16 *>(panel)[row * tl.b + col] = __float2bfloat16_rn(v);
    }
}

// FP32 mode, the update's operand row pr in split FP16: with s = 2^(e - 15)
// (e from the row's slicing: |x| < 2^e), u = (float)x / s (|u| < 2^15, so
// entries down to 2^-29 of the row's largest stay normal FP16 numbers),
// hi = fp16(u), lo = fp16(u - hi), written as the row [hi | lo] of 2b halves;
// s goes to rs[pr].  A row below 2^-100 is treated with e = -100.
template <typename E>
__device__ __forceinline__ void panel_row_f16(const E *x, int b, int e, __half *panel, float *rs, size_t pr)
{
    const int lane = threadIdx.x & 31;
    if (e < -100) e = -100;
    e -= 15;
    const float inv = ldexpf(1.0f, -e);
    __half *row = panel + pr * 2 * (size_t)b;
    for (int c = lane; c < b; c += 32) {
        const float u = (float)x[c] * inv;
        const __half hi = __float2half_rn(u);
        row[c] = hi;
        row[b + c] = __float2half_rn(u - __half2float(hi));
    }
    if (lane == 0) rs[pr] = ldexpf(1.0f, e);
}

// FP32 mode: FP64 band panel rows (m = k+1..k+nrows) -> the BF16 slices of the
// FP64-accurate band updates and the split-FP16 operands of the off-band
// update; one warp per row.
__global__ void __launch_bounds__(256) k_panel_from_f64_split(Tiles tl, int k, void *panel, float *rs,
                                                              __nv_bfloat16 *oz, double *ozs, const DevStatus *st)
{
    if (mfailed(st)) return;
    const int b = tl.b;
    const size_t pr = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);  // panel row
    const int m = k + 1 + (int)(pr / b);
    const double *x = tl.t64(m, k) + (pr % b) * b;
    const int e = slice_row(x, b, oz + pr * b, (size_t)(tl.T - 1) * b * b, ozs + pr);
    panel_row_f16(x, b, e, reinterpret_cast<__half *>(panel), rs, pr);
}

// FP32 mode: solved off-band panel rows (tiles m0 .. T - 1 of column k, FP32)
// -> the BF16 slices of the FP64-accurate band updates and the split-FP16
// operands of the off-band update; one warp per row.
__global__ void __launch_bounds__(256) k_panel_from_f32_split(Tiles tl, int k, int m0, void *panel, float *rs,
                                                              __nv_bfloat16 *oz, double *ozs, const DevStatus *st)
{
    if (mfailed(st)) return;
    const int b = tl.b;
    const size_t pr = (size_t)(m0 - k - 1) * b + (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);  // panel row
    const int m = k + 1 + (int)(pr / b);
    const float *x = tl.t32(m, k) + (pr % b) * b;
    const int e = slice_row_f32(x, b, oz + pr * b, (size_t)(tl.T - 1) * b * b, ozs + pr);
    panel_row_f16(x, b, e, reinterpret_cast<__half *>(panel), rs, pr);
}

// FP32 mode, tensor-core TRSM: the unsolved off-band tiles (m0 .. T - 1, k)
// in the split-TF32 layout [hi | lo] at operand rows (m - k - 1) b + r of pre
// (four consecutive elements per thread).
__global__ void __launch_bounds__(256) k_presplit_a(Tiles tl, int k, int m0, float *__restrict__ pre,
                                                    const DevStatus *st)
{
    if (mfailed(st)) return;
    const int b = tl.b;
    const size_t bb = tl.bb(), total4 = (size_t)(tl.T - m0) * bb / 4, ld = 2 * (size_t)b;
    for (size_t e4 = (size_t)blockIdx.x * 256 + threadIdx.x; e4 < total4; e4 += (size_t)gridDim.x * 256) {
        const size_t e = 4 * e4;
        const int m = m0 + (int)(e / bb);
        const size_t off = e % bb;
        const float4 v = *reinterpret_cast<const float4 *>(tl.t32(m, k) + off);
        float4 hi, lo;
        hi.x = to_tf32(v.x), lo.x = to_tf32(v.x - hi.x);
        hi.y = to_tf32(v.y), lo.y = to_tf32(v.y - hi.y);
        hi.z = to_tf32(v.z), lo.z = to_tf32(v.z - hi.z);
        hi.w = to_tf32(v.w), lo.w = to_tf32(v.w - hi.w);
        float *pa = pre + ((size_t)(m - k - 1) * b + off / b) * ld + off % b;
        *reinterpret_cast<float4 *>(pa) = hi;
        *reinterpret_cast<float4 *>(pa + b) = lo;
    }
}

// W = L_kk^-1 column by column, in FP64: warp w of CTA c solves L w_j = e_j
// for column j = c + gridDim.x w by column-oriented forward substitution:
// with p = e_j, for i = j .. b-1: w_i = p_i / L_ii, then p_r -= L_ri w_i for
// every r > i.  Lane l keeps p_r of the rows r = l + 32 t in registers, so a
// step's critical chain is one shuffle (w_i from its owner lane), one
// multiply and the owner's update of row i + 1; the other rows' updates
// overlap it.  Column i of L_kk is read as row i of LT = L_kk^T, one
// contiguous 256-byte load per 32 rows (reading L_kk itself by columns cost
// 32 cache lines per load).  Each p_r receives its terms in the order of i, so results are
// bitwise reproducible.  Outputs: V_k = W^T (row j of V_k is w_j, the
// upper-triangular inverse the solves use) and W in the split-TF32 layout
// of the tensor-core TRSM (row c: [hi | lo] of (float) W[c][.]).
// NT = b / 32 rows per lane.  Shared memory: (1 + warps) b doubles.
template <int NT>
__global__ void __launch_bounds__(128) k_inv_cols(Tiles tl, int k, const double *__restrict__ LT,
                                                  double *__restrict__ V, float *__restrict__ wsp, const DevStatus *st)
{
    if (mfailed(st)) return;
    extern __shared__ double inv_sm[];
    const int b = tl.b, lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const double *L = tl.t64(k, k);
    double *rinv = inv_sm, *xs = inv_sm + (size_t)(1 + wq) * b;
    for (int i = threadIdx.x; i < b; i += blockDim.x) rinv[i] = 1.0 / L[(size_t)i * b + i];
    for (int i = lane; i < b; i += 32) xs[i] = 0.0;
    __syncthreads();
    const int j = (int)blockIdx.x + (int)gridDim.x * wq;
    double p[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) p[t] = (lane + 32 * t == j) ? 1.0 : 0.0;
    // rows i .. i + D - 1 of LT in registers: a row is loaded D steps before
    // its use, which hides the L2 latency behind D steps of FMAs
    constexpr int D = NT <= 16 ? 4 : (NT <= 24 ? 2 : 1);
    double ring[D][NT];
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
        for (int t = 0; t < NT; ++t) ring[d][t] = (j + d < b) ? LT[(size_t)(j + d) * b + lane + 32 * t] : 0.0;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        if (32 * s + 31 < j) continue;  // rows of this slot lie above j: w = 0 there
        const int ii0 = j > 32 * s ? j - 32 * s : 0;
        for (int ii = ii0; ii < 32; ++ii) {
            const int i = 32 * s + ii;
            double nx[NT];  // row i + D
#pragma unroll
            for (int t = s; t < NT; ++t) nx[t] = (i + D < b) ? LT[(size_t)(i + D) * b + lane + 32 * t] : 0.0;
            const double wi = __shfl_sync(0xffffffffu, p[s], ii) * rinv[i];
            if (lane == 0) xs[i] = wi;
#pragma unroll
            for (int t = s; t < NT; ++t)
                if (lane + 32 * t > i) p[t] = fma(-ring[0][t], wi, p[t]);
#pragma unroll
            for (int t = s; t < NT; ++t) {
#pragma unroll
                for (int d = 0; d + 1 < D; ++d) ring[d][t] = ring[d + 1][t];
                ring[D - 1][t] = nx[t];
            }
        }
    }
    __syncwarp();
    double *Vj = V + (size_t)k * tl.bb() + (size_t)j * b;
    const size_t ld2 = 2 * (size_t)b;
    for (int c = lane; c < b; c += 32) {
        const double x = xs[c];
        Vj[c] = x;
        const float v = (float)x, hi = to_tf32(v), lo = to_tf32(v - hi);
        float *pw = wsp + (size_t)c * ld2 + j;
        pw[0] = hi;
        pw[b] = lo;
    }
}

// LT = L_kk^T (32 x 32 blocks through shared memory), so that the inversion
// reads a column of L_kk as one contiguous row.
__global__ void __launch_bounds__(256) k_transpose_diag(Tiles tl, int k, double *__restrict__ LT, const DevStatus *st)
{
    __shared__ double blk[32][33];
    if (mfailed(st)) return;
    const int b = tl.b, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r0 = 32 * (int)blockIdx.y, c0 = 32 * (int)blockIdx.x;
    const double *L = tl.t64(k, k);
    for (int r = ty; r < 32; r += 8) blk[r][tx] = L[(size_t)(r0 + r) * b + c0 + tx];
    __syncthreads();
    for (int r = ty; r < 32; r += 8) LT[(size_t)(c0 + r) * b + r0 + tx] = blk[tx][r];
}

cudaError_t launch_inv_cols(const Tiles &tl, int k, double *LT, double *V, float *wsp, const DevStatus *st,
                            cudaStream_t s, KernelTimer *kt)
{
    const int b = tl.b;
    EGS_LAUNCH(kt, KC_TRSM, s,
               k_transpose_diag<<<dim3((unsigned)(b / 32), (unsigned)(b / 32)), 256, 0, s>>>(tl, k, LT, st));
    const unsigned grid = (unsigned)(b / 4);
    const size_t sm = (size_t)5 * b * sizeof(double);
    switch (b / 32) {
    case 8: EGS_LAUNCH(kt, KC_TRSM, s, k_inv_cols<8><<<grid, 128, sm, s>>>(tl, k, LT, V, wsp, st)); break;
    case 16: EGS_LAUNCH(kt, KC_TRSM, s, k_inv_cols<16><<<grid, 128, sm, s>>>(tl, k, LT, V, wsp, st)); break;
    case 24: EGS_LAUNCH(kt, KC_TRSM, s, k_inv_cols<24><<<grid, 128, sm, s>>>(tl, k, LT, V, wsp, st)); break;
    case 32: EGS_LAUNCH(kt, KC_TRSM, s, k_inv_cols<32><<<grid, 128, sm, s>>>(tl, k, LT, V, wsp, st)); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// FP64 band panel tiles (m = k+1..k+nrows) -> operand format.
template <int FMT>
__global__ void __launch_bounds__(256) k_panel_from_f64(Tiles tl, int k, int nrows, void *panel, const DevStatus *st)
{
    if (mfailed(st)) return;
    const size_t bb = tl.bb();
    const size_t total = (size_t)nrows * bb;
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (size_t)gridDim.x * 256) {
        const int t = (int)(e / bb);
        const size_t off = e % bb;
        const int m = k + 1 + t;
        panel_store<FMT>(panel, tl, (size_t)(m - k - 1) * tl.b + off / tl.b, (int)(off % tl.b),
                         (float)tl.t64(m, k)[off]);
    }
}

// FP64 TRSM of the band rows of step k (tiles (k+1 .. k+nb, k)): X L_kk^T = A,
// solved in place.  A CTA keeps kTbR rows of one tile in shared memory and
// sweeps the 32-column blocks of L_kk: block j first subtracts the solved
// columns, X[:, 0:32j] L[32j:32j+32, 0:32j]^T, one 32 x 32 chunk of L at a
// time (staged transposed in shared memory while the next chunk is loaded
// into registers; two warps per row, each over half of a chunk), then one
// warp per row solves the 32 x 32 diagonal block by column-oriented
// substitution (a shuffle, a multiplication by 1 / L_ii and an FMA per
// column).  b / kTbR CTAs per tile spread the b^3 / 2 FMA of a tile over the
// GPU; the chain of the FP64 band is latency-bound, and this solve sits on it
// once per step.
constexpr int kTbR = 4;
static_assert(kTbR * 64 == 256, "two warps per row of the CTA");
__global__ void __launch_bounds__(256) k_trsm_band_f64(Tiles tl, int k, const DevStatus *st)
{
    extern __shared__ double tb_xs[];  // kTbR x b: the CTA's rows
    __shared__ double LcT[2][32][33];  // chunk (j, i) transposed: LcT[cc][cr] = L[32j + cr][32i + cc]
    __shared__ double part[2][kTbR][32];
    __shared__ double rdg[1024];  // 1 / L_ii
    if (mfailed(st)) return;
    const int b = tl.b, nblk = b >> 5, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid >> 6, h = (tid >> 5) & 1;  // row of the CTA, half of a chunk
    double *X = tl.t64(k + 1 + (int)blockIdx.y, k) + (size_t)blockIdx.x * kTbR * b;
    const double *L = tl.t64(k, k);
    for (int e = tid; e < kTbR * b; e += 256) tb_xs[e] = X[e];
    for (int e = tid; e < b; e += 256) rdg[e] = 1.0 / L[(size_t)e * b + e];
    double reg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) reg[q] = L[(size_t)((tid >> 5) + 8 * q) * b + lane];  // chunk (0, 0)
    double acc = 0.0;
    int j = 0, i = 0, buf = 0;
    for (;;) {
#pragma unroll
        for (int q = 0; q < 4; ++q) LcT[buf][lane][(tid >> 5) + 8 * q] = reg[q];
        int jn = j, in = i + 1;
        if (in > jn) {
            ++jn;
            in = 0;
        }
        if (jn < nblk) {
#pragma unroll
            for (int q = 0; q < 4; ++q) reg[q] = L[(size_t)(32 * jn + (tid >> 5) + 8 * q) * b + 32 * in + lane];
        }
        __syncthreads();
        if (i < j) {
            const double *xr = tb_xs + (size_t)r * b + 32 * i + 16 * h;
#pragma unroll
            for (int l = 0; l < 16; ++l) acc = fma(xr[l], LcT[buf][16 * h + l][lane], acc);
        } else {
            part[h][r][lane] = acc;
            acc = 0.0;
            __syncthreads();
            if (warp < kTbR) {
                double *xj = tb_xs + (size_t)warp * b + 32 * j;
                double v = xj[lane] - (part[0][warp][lane] + part[1][warp][lane]);
                for (int l = 0; l < 32; ++l) {
                    // every lane forms x_l (a warp-wide FP64 instruction costs
                    // the same with one lane active or all 32)
                    const double x = __shfl_sync(0xffffffffu, v, l) * rdg[32 * j + l];
                    const double u = fma(-x, LcT[buf][l][lane], v);
                    v = lane > l ? u : (lane == l ? x : v);
                }
                xj[lane] = v;
            }
        }
        j = jn;
        i = in;
        buf ^= 1;
        if (j >= nblk) break;
    }
    __syncthreads();
    for (int e = tid; e < kTbR * b; e += 256) X[e] = tb_xs[e];
}

cudaError_t launch_trsm_band_f64(const Tiles &tl, int k, int nb, const DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    if (nb <= 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(k_trsm_band_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, kTbR * 1024 * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    EGS_LAUNCH(kt, KC_TRSM, s,
               k_trsm_band_f64<<<dim3((unsigned)(tl.b / kTbR), (unsigned)nb), 256, (size_t)kTbR * tl.b * sizeof(double),
                                 s>>>(tl, k, st));
    return cudaGetLastError();
}

// L_kk rounded to FP32 once per step for the FP32 TRSM of the TF32 / BF16
// modes (it reads L_kk many times; a conversion from FP64 runs on the FP64
// pipe, 2 per clock per SM on GB300).
__global__ void __launch_bounds__(256) k_l32_from_f64(Tiles tl, int k, float *__restrict__ l32, const DevStatus *st)
{
    if (mfailed(st)) return;
    const double *L = tl.t64(k, k);
    const size_t bb = tl.bb();
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < bb; e += (size_t)gridDim.x * 256) l32[e] = (float)L[e];
}

// TRSM of the FP32 panel rows m = m0 + blockIdx.x (TF32 / BF16 modes):
// X L_kk^T = A_mk in FP32 (L_kk rounded to FP32, l32), 64 rows per CTA,
// 32-column blocks; the result
// overwrites A_mk and is written to the panel buffer.  The GEMM-style part
// keeps 4 rows x 2 columns per thread with the operands transposed in shared
// memory (one 16-byte and one 8-byte shared load per 8 FMAs).  The kernel is
// latency bound; 80 registers let three CTAs share an SM (802 -> 687 us per
// launch at n = 32,768; four CTAs need 64 registers and spill).
template <int FMT>
__global__ void __launch_bounds__(256, 3) k_trsm_panel_f32(Tiles tl, int k, int m0, const float *__restrict__ L,
                                                        void *panel, __nv_bfloat16 *oz, double *ozs, const DevStatus *st)
{
    if (mfailed(st)) return;
    const int b = tl.b;
    const int m = m0 + (int)blockIdx.x;
    const int r0 = (int)blockIdx.y * 64;
    float *A = tl.t32(m, k) + (size_t)r0 * b;
    const size_t prow0 = (size_t)(m - k - 1) * b + r0;
    __shared__ __align__(16) float Xt[16][64];   // [l][row]
    __shared__ __align__(16) float Lt[16][32];   // [l][col]
    __shared__ float Ab[64][33];
    __shared__ float Ld[32][33];
    const int tid = threadIdx.x;
    const int tc = tid & 15, tr = tid >> 4;      // columns 2 tc, 2 tc + 1; rows 4 tr .. 4 tr + 3
    for (int c0 = 0; c0 < b; c0 += 32) {
        float acc[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[i][j] = A[(size_t)(4 * tr + i) * b + c0 + 2 * tc + j];
        for (int p = 0; p < c0; p += 16) {
            for (int e = tid; e < 64 * 16; e += 256) {
                const int r = e >> 4, l = e & 15;
                Xt[l][r] = A[(size_t)r * b + p + l];
            }
            for (int e = tid; e < 32 * 16; e += 256) {
                const int c = e >> 4, l = e & 15;
                Lt[l][c] = L[(size_t)(c0 + c) * b + p + l];
            }
            __syncthreads();
#pragma unroll
            for (int l = 0; l < 16; ++l) {
                const float4 x = *reinterpret_cast<const float4 *>(&Xt[l][4 * tr]);
                const float2 lv = *reinterpret_cast<const float2 *>(&Lt[l][2 * tc]);
                acc[0][0] = fmaf(-x.x, lv.x, acc[0][0]);
                acc[0][1] = fmaf(-x.x, lv.y, acc[0][1]);
                acc[1][0] = fmaf(-x.y, lv.x, acc[1][0]);
                acc[1][1] = fmaf(-x.y, lv.y, acc[1][1]);
                acc[2][0] = fmaf(-x.z, lv.x, acc[2][0]);
                acc[2][1] = fmaf(-x.z, lv.y, acc[2][1]);
                acc[3][0] = fmaf(-x.w, lv.x, acc[3][0]);
                acc[3][1] = fmaf(-x.w, lv.y, acc[3][1]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) Ab[4 * tr + i][2 * tc + j] = acc[i][j];
        for (int e = tid; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            Ld[r][c] = (c <= r) ? L[(size_t)(c0 + r) * b + c0 + c] : 0.0f;
        }
        __syncthreads();
        if (tid < 64) {
            for (int j = 0; j < 32; ++j) {
                float s = Ab[tid][j];
                for (int l = 0; l < j; ++l) s = fmaf(-Ab[tid][l], Ld[j][l], s);
                Ab[tid][j] = s / Ld[j][j];
            }
        }
        __syncthreads();
        for (int e = tid; e < 64 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            const float v = Ab[r][c];
            const size_t off = (size_t)r * b + c0 + c;
            A[off] = v;
            panel_store<FMT>(panel, tl, prow0 + r, c0 + c, v);
        }
        __syncthreads();
    }
    if (FMT == 3) {
        // slices of the 64 solved rows for the FP64-accurate band updates
        // (re-read from L1/L2; one warp per row)
        const size_t R = (size_t)(tl.T - 1) * b;
        for (int rr = tid >> 5; rr < 64; rr += 8)
            slice_row_f32(A + (size_t)rr * b, b, oz + (prow0 + rr) * b, R * b, ozs + prow0 + rr);
    }
}

// Backward substitution on diagonal tile k: L_kk^T x = r in place (b threads).
__global__ void __launch_bounds__(1024) k_trsv_diag_T(Tiles tl, int k, double *__restrict__ v, const DevStatus *st)
{
    if (mfailed(st)) return;
    trsv_bwd_tile(tl.t64(k, k), tl.b, v + (size_t)k * tl.b);
}

// r_j -= L_kj^T x_k for j < k (x_k read from xsrc, which may equal v).
// grid = (k, b/64).
__global__ void __launch_bounds__(256) k_gemv_T(Tiles tl, int k, const double *xsrc, double *v, const DevStatus *st)
{
    if (mfailed(st)) return;
    gemv_T_cols(tl, k, (int)blockIdx.x, (int)blockIdx.y * 64, xsrc + (size_t)k * tl.b, v + (size_t)blockIdx.x * tl.b);
}

// V_k = L_kk^-T for every diagonal tile k = blockIdx.x: 16 rows of V_k per
// CTA, each the solution of x L_kk^T = e_r (trsm_rows on identity rows; the
// columns before the row's 32-column block are zero and skipped).  V_k is
// upper triangular, so y = L_kk^-1 r = V_k^T r and x = L_kk^-T r = V_k r
// become matrix-vector products spread over many SMs instead of a serial
// substitution on one.
__global__ void __launch_bounds__(256) k_inv_diag(Tiles tl, double *__restrict__ V, const DevStatus *st)
{
    if (mfailed(st)) return;
    const int b = tl.b, k = (int)blockIdx.x, r0 = (int)blockIdx.y * 16;
    double *X = V + (size_t)k * tl.bb() + (size_t)r0 * b;
    for (int e = threadIdx.x; e < 16 * b; e += 256) X[e] = (e / b + r0 == e % b) ? 1.0 : 0.0;
    __syncthreads();
    trsm_rows<16>(tl.t64(k, k), b, X, b, b, (r0 / 32) * 32);
}

// partials[k] = sum_i log L_kk[i][i] (fixed-order tree).
__global__ void __launch_bounds__(256) k_logdet_tiles(Tiles tl, double *__restrict__ partials, const DevStatus *st)
{
    if (mfailed(st)) return;
    __shared__ double red[256];
    const int b = tl.b, k = (int)blockIdx.x;
    const double *L = tl.t64(k, k);
    double a = 0.0;
    for (int i = threadIdx.x; i < b; i += 256) a += log(L[(size_t)i * b + i]);
    const double tot = block_sum(a, red);
    if (threadIdx.x == 0) partials[k] = tot;
}

// out_k = V_k^T rhs_k (= L_kk^-1 rhs_k): 8 columns per CTA (b / 8 CTAs).  The
// CTA stages its column strip of V_k 256 rows at a time in shared memory
// (rows r <= c only: V_k is upper triangular), every load of a chunk in
// flight at once, then 32 row groups x 8 columns multiply and reduce in a
// fixed order.
__global__ void __launch_bounds__(256) k_fwd_inv(const double *__restrict__ V, int b, int k,
                                                 const double *__restrict__ rhs, double *__restrict__ out,
                                                 const DevStatus *st)
{
    if (mfailed(st)) return;
    __shared__ double vs[256][8];
    __shared__ double red[32][9];
    const double *Vk = V + (size_t)k * b * b;
    const double *xk = rhs + (size_t)k * b;
    const int c0 = (int)blockIdx.x * 8, tx = threadIdx.x & 7, g = threadIdx.x >> 3;
    const int rend = c0 + 8;  // rows beyond the strip's last column are zero
    double sacc = 0.0;
    for (int r0 = 0; r0 < rend; r0 += 256) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = r0 + g + 32 * i;
            vs[g + 32 * i][tx] = r < rend ? Vk[(size_t)r * b + c0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = r0 + g + 32 * i;
            if (r < rend) sacc = fma(vs[g + 32 * i][tx], xk[r], sacc);
        }
        __syncthreads();
    }
    red[g][tx] = sacc;
    __syncthreads();
    if (g == 0) {
        double t = red[0][tx];
#pragma unroll
        for (int q = 1; q < 32; ++q) t += red[q][tx];
        out[(size_t)k * b + c0 + tx] = t;
    }
}
// out_k = V_k rhs_k (= L_kk^-T rhs_k): one row per warp (b / 8 CTAs), columns
// c >= r, fixed shuffle tree.
__global__ void __launch_bounds__(256) k_bwd_inv(const double *__restrict__ V, int b, int k,
                                                 const double *__restrict__ rhs, double *__restrict__ out,
                                                 const DevStatus *st)
{
    if (mfailed(st)) return;
    __shared__ double xs[1024];
    const double *Vk = V + (size_t)k * b * b;
    for (int c = threadIdx.x; c < b; c += 256) xs[c] = rhs[(size_t)k * b + c];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (int)blockIdx.x * 8 + warp;
    const double *row = Vk + (size_t)r * b;
    double sacc = 0.0;
    for (int c = (r & ~31) + lane; c < b; c += 32) sacc = fma(row[c], xs[c], sacc);  // row[c] = 0 for c < r
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
    if (lane == 0) out[(size_t)k * b + r] = sacc;
}

__global__ void k_axpy(double *__restrict__ x, const double *__restrict__ d, int64_t npad, const DevStatus *st)
{
    if (mfailed(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npad) x[i] += d[i];
}

__global__ void k_copy(double *__restrict__ dst, const double *__restrict__ src, int64_t npad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npad) dst[i] = src[i];
}

// l from log-det partials, quad0 = y.y (y = L^-1 z) and quad = z.x (fixed order).
__global__ void __launch_bounds__(1024) k_finalize_mixed(const double *__restrict__ partials, int T,
                                                         const double *__restrict__ zp, const double *__restrict__ x,
                                                         const double *__restrict__ y, int64_t npad, int64_t n,
                                                         int refined, DevStatus *st)
{
    __shared__ double red[1024];
    const int tid = threadIdx.x;
    double a = 0.0, q0 = 0.0, q = 0.0;
    for (int t = tid; t < T; t += 1024) a += partials[t];
    for (int64_t i = tid; i < npad; i += 1024) {
        q = fma(zp[i], x[i], q);
        q0 = fma(y[i], y[i], q0);
    }
    double vals[3] = {a, q0, q};
    double tot[3];
    for (int v = 0; v < 3; ++v) {
        red[tid] = vals[v];
        __syncthreads();
        for (int s = 512; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        tot[v] = red[0];
        __syncthreads();
    }
    if (tid == 0) {
        if (mfailed(st)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            st->result[0] = st->result[1] = st->result[2] = st->result[3] = nan;
        } else {
            const double logdet = 2.0 * tot[0];
            const double quad = refined ? tot[2] : tot[1];
            st->result[0] = -0.5 * quad - 0.5 * logdet - 0.5 * (double)n * 1.8378770664093454836;
            st->result[1] = logdet;
            st->result[2] = quad;
            st->result[3] = tot[1];
        }
    }
}

}  // namespace

// L^T x = v in place on v (T b doubles): block column substitution from the
// last tile, FP64 arithmetic (FP32 off-band tiles are read as FP32).
cudaError_t backward_solve(const Tiles &tl, double *v, const DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    for (int k = tl.T - 1; k >= 0; --k) {
        EGS_LAUNCH(kt, KC_TRSV, s, k_trsv_diag_T<<<1, tl.b, 0, s>>>(tl, k, v, st));
        if (k > 0)
            EGS_LAUNCH(kt, KC_TRSV, s, k_gemv_T<<<dim3((unsigned)k, (unsigned)(tl.b / 64)), 256, 0, s>>>(tl, k, v, v, st));
    }
    return cudaGetLastError();
}

namespace {

// The factorisation with one step of lookahead.  The FP64 chain of step k
// (POTRF, the band TRSM, the band rows' operands, then the FP64 band x band
// update) runs on a side stream; the main stream runs the TRSM of the
// off-band panel on the whole GPU and the tensor-core update of column k + 1,
// signals the side stream, and updates the rest of the trailing matrix
// (leaving a few SMs free) while the next chain runs.  Diagonal tile k + 1
// is final once the chain's own band x band update of step k is done (every
// other update of column k + 1 writes tiles below it), so POTRF(k + 1) does
// not wait for the main stream: only the band TRSM of step k + 1, whose rows
// column k + 1's other updates write, waits for its signal.  In the FP32 mode
// the chain also inverts L_kk right after POTRF(k) (a latency-bound kernel
// kept off the main stream), and the main stream's off-band TRSM through
// L_kk^-1 starts once that is done, beside the chain's band TRSM.  Panels,
// W (and in FP32 mode the slices) alternate between two buffers.
template <int FMT>
cudaError_t factor_mixed(const MixedBuffers &mb, const CUtensorMap *ma, const CUtensorMap *mbm, const CUtensorMap *ma3,
                         const CUtensorMap &mc, const CUtensorMap (*moz)[2], const CUtensorMap *mw, DevStatus *st,
                         cudaStream_t s, KernelTimer *kt)
{
    const Tiles &tl = mb.tl;
    const int T = tl.T, b = tl.b;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_col = nullptr, ev_diag = nullptr;
    // The chain gates the next step, so its kernels take the SMs that the
    // main stream's kernels free first: the side stream runs at the highest
    // priority (otherwise each step's POTRF waits for the whole slice-product
    // launch ahead of it to drain).
    int prio_least = 0, prio_greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_col, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_diag, cudaEventDisableTiming);
    if (e == cudaSuccess)  // the one-launch diagonal POTRFs' counters
        e = cudaMemsetAsync(mb.pctr, 0, (size_t)T * potrf_diag_scratch_words(b) * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaEventRecord(ev_col, s);  // the side stream starts after prior work on s
    KernelTimer *kts = kt;  // side-stream kernels are timed with events on the side stream
    for (int k = 0; k < T && e == cudaSuccess; ++k) {
        if (kt) kt->step = k;
        const int nb = (tl.band - 1 < T - k - 1) ? tl.band - 1 : T - k - 1;  // FP64 rows below k
        const int nf = T - k - 1 - nb;                                       // FP32 rows
        void *panel = mb.panel[k & 1];
        __nv_bfloat16 *oz = (__nv_bfloat16 *)mb.oz[k & 1];
        double *ozs = mb.ozs[k & 1];
        // ---- chain of step k on the side stream: POTRF (tile k was final
        // after the chain's band x band update of step k - 1), then, once
        // the main stream has updated column k, the FP64 band TRSM and the
        // band rows' operands; then (after signalling the main stream) the
        // FP64 band x band update.  At k = 0 ev_col marks the work on s
        // before the call (Sigma generation).
        if (k == 0) e = cudaStreamWaitEvent(side, ev_col, 0);
        if (e == cudaSuccess)
            e = launch_potrf_diag(tl, k, st, side, kts, mb.pctr + (size_t)k * potrf_diag_scratch_words(b));
        // FP32 mode: W = L_kk^-1 (and V_k = W^T for the solves) for the main
        // stream's off-band TRSM, off the main stream
        float *wsp = mb.wsp + (size_t)(k & 1) * 2 * tl.bb();
        if (e == cudaSuccess && FMT == 3) e = launch_inv_cols(tl, k, mb.lt, mb.vinv, wsp, st, side, kts);
        if (e == cudaSuccess) e = cudaEventRecord(ev_diag, side);
        if (e == cudaSuccess && k > 0) e = cudaStreamWaitEvent(side, ev_col, 0);
        if (e == cudaSuccess && k + 1 < T) {
            if (nf > 0 && FMT != 3)
                EGS_LAUNCH(kts, KC_TRSM, side,
                           k_l32_from_f64<<<(unsigned)((tl.bb() + 255) / 256 < 1024 ? (tl.bb() + 255) / 256 : 1024), 256,
                                            0, side>>>(tl, k, mb.l32, st));
            e = launch_trsm_band_f64(tl, k, nb, st, side, kts);
            if (e == cudaSuccess && nb > 0) {
                if (FMT == 3) {
                    EGS_LAUNCH(kts, KC_TRSM, side,
                               k_panel_from_f64_split<<<(unsigned)((size_t)nb * b / 8), 256, 0, side>>>(
                                   tl, k, panel, mb.rs[k & 1], oz, ozs, st));
                } else {
                    const size_t total = (size_t)nb * tl.bb();
                    const unsigned blocks = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
                    EGS_LAUNCH(kts, KC_TRSM, side,
                               k_panel_from_f64<FMT><<<blocks, 256, 0, side>>>(tl, k, nb, panel, st));
                }
            }
            if (e == cudaSuccess) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_panel, side);
        // updates whose two operands are FP64 band tiles stay FP64-accurate
        // (they carry the nearest-neighbour entries that set the diagonal
        // pivots): on DFMA, or in the FP32 mode as exact slice products;
        // their outputs are read by nothing else at this step
        if (e == cudaSuccess && k + 1 < T) {
            if (FMT == 3)  // FP32 mode: from the band rows' exact slices on tcgen05
                e = launch_band_band_ozaki(moz[k & 1][0], moz[k & 1][1], tl, k, nb, ozs, mb.err, side, kts);
            else
                e = launch_update_f64(tl, k, (int64_t)nb * (nb + 1) / 2, st, side, kts, KC_UPDATE64);
        }
        if (k + 1 == T || e != cudaSuccess) break;
        // ---- step k on the main stream: the off-band TRSM (whole GPU),
        // column k + 1, signal, then the rest
        e = cudaStreamWaitEvent(s, FMT == 3 ? ev_diag : ev_panel, 0);
        if (FMT == 3) {
            // X = A W^T on the tensor cores with W = L_kk^-1 from the chain
            // stream: the unsolved tiles are split into the spare panel
            // buffer (free until the next step's chain writes its band rows,
            // after column k + 1 below), the product overwrites them, and the solved
            // rows are split into this step's panel and slices
            const int m0 = k + 1 + nb;
            if (e == cudaSuccess && nf > 0) {
                const size_t total4 = (size_t)nf * tl.bb() / 4;
                const unsigned g4 = (unsigned)((total4 + 255) / 256 < 2048 ? (total4 + 255) / 256 : 2048);
                EGS_LAUNCH(kt, KC_TRSM, s,
                           k_presplit_a<<<g4, 256, 0, s>>>(tl, k, m0, (float *)mb.panel[(k + 1) & 1], st));
                e = launch_trsm_tc(ma3[(k + 1) & 1], mw[k & 1], mc, tl, k, m0, mb.err, s, kt);
                if (e == cudaSuccess)
                    EGS_LAUNCH(kt, KC_TRSM, s,
                               k_panel_from_f32_split<<<(unsigned)((size_t)nf * b / 8), 256, 0, s>>>(
                                   tl, k, m0, panel, mb.rs[k & 1], oz, ozs, st));
            }
        } else if (e == cudaSuccess && nf > 0) {
            EGS_LAUNCH(kt, KC_TRSM, s,
                       k_trsm_panel_f32<FMT><<<dim3((unsigned)nf, (unsigned)(b / 64)), 256, 0, s>>>(
                           tl, k, k + 1 + nb, mb.l32, panel, oz, ozs, st));
        }
        // the band rows' operands (and slices) come from the chain
        if (e == cudaSuccess && FMT == 3) e = cudaStreamWaitEvent(s, ev_panel, 0);
        // FP32 mode: band outputs with an FP32 operand by exact slices
        if (e == cudaSuccess && FMT == 3)
            e = launch_band_out_ozaki(moz[k & 1][0], moz[k & 1][1], tl, mb.xband, k, k + 1, 1, ozs, mb.err, s, kt);
        // FP32 mode: the off-band update in split FP16 (fmt 4) from the scaled rows
        const int ufmt = FMT == 3 ? 4 : FMT;
        const float *urs = FMT == 3 ? mb.rs[k & 1] : nullptr;
        if (e == cudaSuccess)
            e = launch_update_tc(ma[k & 1], mbm[k & 1], mc, ufmt, tl, k, mb.err, s, kt, 1, urs, mb.xband);
        if (e == cudaSuccess) e = cudaEventRecord(ev_col, s);
        if (e == cudaSuccess && FMT == 3)
            e = launch_band_out_ozaki(moz[k & 1][0], moz[k & 1][1], tl, mb.xband, k, k + 2, T - k - 2, ozs, mb.err, s,
                                      kt);
        if (e == cudaSuccess)
            e = launch_update_tc(ma[k & 1], mbm[k & 1], mc, ufmt, tl, k, mb.err, s, kt, 2, urs, mb.xband);
    }
    if (kt) kt->step = -1;
    if (e == cudaSuccess) e = cudaEventRecord(ev_panel, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_panel, 0);  // join the side stream
    // destroying a stream or event with work still pending is legal: the
    // resources are released once that work completes, and s already waits
    // for it through ev_panel
    if (side) cudaStreamDestroy(side);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (ev_col) cudaEventDestroy(ev_col);
    if (ev_diag) cudaEventDestroy(ev_diag);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

// out = L^-1 rhs with the inverted diagonal tiles (rhs is overwritten).
cudaError_t forward_solve_inv(const Tiles &tl, const double *V, double *rhs, double *out, const DevStatus *st,
                              cudaStream_t s, KernelTimer *kt)
{
    for (int k = 0; k < tl.T; ++k) {
        EGS_LAUNCH(kt, KC_TRSV, s, k_fwd_inv<<<(unsigned)(tl.b / 8), 256, 0, s>>>(V, tl.b, k, rhs, out, st));
        cudaError_t e = launch_gemv_panel(tl, k, out, rhs, st, s, kt);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// out = L^-T rhs with the inverted diagonal tiles (rhs is overwritten).
cudaError_t backward_solve_inv(const Tiles &tl, const double *V, double *rhs, double *out, const DevStatus *st,
                               cudaStream_t s, KernelTimer *kt)
{
    for (int k = tl.T - 1; k >= 0; --k) {
        EGS_LAUNCH(kt, KC_TRSV, s, k_bwd_inv<<<(unsigned)(tl.b / 8), 256, 0, s>>>(V, tl.b, k, rhs, out, st));
        if (k > 0)
            EGS_LAUNCH(kt, KC_TRSV, s,
                       k_gemv_T<<<dim3((unsigned)k, (unsigned)(tl.b / 64)), 256, 0, s>>>(tl, k, out, rhs, st));
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_loglik_mixed(const double *X, const double *Y, const double *z, int64_t n, const egs_matern_params &P,
                             int fmt, int refine, const MixedBuffers &mb, DevStatus *st, cudaStream_t s, KernelTimer *kt,
                             cudaEvent_t *ev)
{
    const Tiles &tl = mb.tl;
    const int b = tl.b, T = tl.T;
    const int64_t npad = (int64_t)T * b;
    const unsigned vb = (unsigned)((npad + 255) / 256);
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_matern_tiles(X, Y, n, tl, P, s, kt, mb.mtab);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    // update maps (FP32 mode: split FP16 over the panel buffers) and, in the
    // FP32 mode, split-TF32 maps over the same buffers for the TRSM's operand
    CUtensorMap ma[2], mbm[2], ma3[2], mb3, mc, moz[2][2];
    const int ufmt = fmt == 3 ? 4 : fmt;
    e = make_panel_maps(mb.panel[0], ufmt, b, T, &ma[0], &mbm[0]);
    if (e == cudaSuccess) e = make_panel_maps(mb.panel[1], ufmt, b, T, &ma[1], &mbm[1]);
    for (int i = 0; i < 2 && e == cudaSuccess && fmt == 3; ++i) e = make_panel_maps(mb.panel[i], 3, b, T, &ma3[i], &mb3);
    if (e == cudaSuccess) e = make_offband_map(tl.f32, b, Tiles::f32_tiles(T, tl.band), &mc);
    for (int i = 0; i < 2 && e == cudaSuccess && fmt == 3; ++i) e = make_ozaki_maps(mb.oz[i], b, T, &moz[i][0], &moz[i][1]);
    if (e != cudaSuccess) return e;
    CUtensorMap mw[2];
    for (int i = 0; i < 2 && e == cudaSuccess && fmt == 3; ++i)
        e = make_trsm_w_map(mb.wsp + (size_t)i * 2 * tl.bb(), b, &mw[i]);
    if (e != cudaSuccess) return e;
    if (fmt == 3) e = factor_mixed<3>(mb, ma, mbm, ma3, mc, moz, mw, st, s, kt);
    else if (fmt == 2) e = factor_mixed<2>(mb, ma, mbm, ma3, mc, moz, nullptr, st, s, kt);
    else e = factor_mixed<1>(mb, ma, mbm, ma3, mc, moz, nullptr, st, s, kt);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], s);
    // V_k = L_kk^-T for every diagonal tile (FP32 mode: computed during the
    // factorisation) and the log-det partials, then res = L^-1 z (kept for
    // y.y), x = L^-T res
    if (fmt != 3)
        EGS_LAUNCH(kt, KC_TRSV, s, k_inv_diag<<<dim3((unsigned)T, (unsigned)(b / 16)), 256, 0, s>>>(tl, mb.vinv, st));
    EGS_LAUNCH(kt, KC_TRSV, s, k_logdet_tiles<<<(unsigned)T, 256, 0, s>>>(tl, mb.partials, st));
    e = launch_pad_vector(z, n, mb.zp, npad, s, kt);
    if (e != cudaSuccess) return e;
    EGS_LAUNCH(kt, KC_OTHER, s, k_copy<<<vb, 256, 0, s>>>(mb.y, mb.zp, npad));
    e = forward_solve_inv(tl, mb.vinv, mb.y, mb.res, st, s, kt);
    if (e != cudaSuccess) return e;
    EGS_LAUNCH(kt, KC_OTHER, s, k_copy<<<vb, 256, 0, s>>>(mb.d, mb.res, npad));
    e = backward_solve_inv(tl, mb.vinv, mb.d, mb.x, st, s, kt);
    if (e != cudaSuccess) return e;
    for (int it = 0; it < refine; ++it) {
        // d = z - Sigma x with Sigma regenerated tile by tile (no stored copy)
        e = launch_residual_regen(X, Y, n, b, T, P, mb.mtab, mb.x, mb.zp, mb.slots, mb.d, st, s, kt);
        if (e != cudaSuccess) return e;
        // correction: y = L^-1 d, rows = L^-T y (rows is free once d is formed)
        e = forward_solve_inv(tl, mb.vinv, mb.d, mb.y, st, s, kt);
        if (e != cudaSuccess) return e;
        e = backward_solve_inv(tl, mb.vinv, mb.y, mb.rows, st, s, kt);
        if (e != cudaSuccess) return e;
        EGS_LAUNCH(kt, KC_OTHER, s, k_axpy<<<vb, 256, 0, s>>>(mb.x, mb.rows, npad, st));
    }
    EGS_LAUNCH(kt, KC_OTHER, s,
               k_finalize_mixed<<<1, 1024, 0, s>>>(mb.partials, T, mb.zp, mb.x, mb.res, npad, n, refine > 0 ? 1 : 0,
                                                   st));
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

}  // namespace egs
