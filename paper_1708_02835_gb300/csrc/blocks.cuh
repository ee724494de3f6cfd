// FP64 dense-block device routines shared by the single-problem and the
// batched drivers (included by several translation units; no relocatable
// device code needed).  Every routine is executed by a whole CTA of 256
// threads unless stated otherwise.
#pragma once
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
// Cholesky of a 64 x 64 block at A (row stride ld) held in shared memory for
// the whole factorisation (one global read and one write of the block): one
// CTA of 256 threads, right-looking over four 16-column panels -- warp 0
// factors the 16 x 16 diagonal block with warp synchronisation only, each row
// below it is solved by one thread, and the trailing lower triangle takes a
// rank-16 update (one 16-term dot product per entry) -- so the block needs 12
// CTA barriers, and its FP64 work is mostly independent FMAs.  Pivots are
// applied through 1 / sqrt(d) (one reciprocal square root per column, then
// multiplications).  A pivot that is not positive records row0 + its row in
// st->fail_index and returns false; the strict upper triangle is zeroed.
// The same routine serves NB = 32.
// ---------------------------------------------------------------------------
template <int NB>
struct PotrfSmem {
    double S[NB][NB + 1];
    double rd[NB];  // 1 / L_jj
    int fail_j;
};
using Potrf64Smem = PotrfSmem<64>;

// NB x NB block (NB = 32 or 64), as described above.
template <int NB>
__device__ __forceinline__ bool potrf_smem_s(PotrfSmem<NB> &sm, double *A, int ld, int64_t row0, DevStatus *st)
{
    double(&S)[NB][NB + 1] = sm.S;
    int &fail_j = sm.fail_j;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) fail_j = -1;
    for (int e = tid; e < NB * NB; e += 256) {
        const int i = e / NB, j = e % NB;
        S[i][j] = (j <= i) ? A[(size_t)i * ld + j] : 0.0;
    }
    __syncthreads();
    for (int p0 = 0; p0 < NB; p0 += kPW) {
        // 1. the 16 x 16 diagonal block, column by column, by warp 0 (lane i < 16 owns row p0 + i)
        if (tid < 32) {
            for (int j = 0; j < kPW; ++j) {
                // every lane forms 1 / sqrt(d) (a warp-wide FP64 instruction
                // costs the same for one lane or 32), so the column is scaled
                // by a multiplication instead of a division
                const double d = S[p0 + j][p0 + j];
                if (!(d > 0.0)) {
                    if (lane == 0) fail_j = p0 + j;
                    break;
                }
                const double rs = rsqrt(d);
                __syncwarp();
                if (lane == j) {
                    S[p0 + j][p0 + j] = d * rs;
                    sm.rd[p0 + j] = rs;
                }
                if (lane > j && lane < kPW) S[p0 + lane][p0 + j] *= rs;
                __syncwarp();
                if (lane > j && lane < kPW) {
                    const double lij = S[p0 + lane][p0 + j];
                    for (int l = j + 1; l <= lane; ++l) S[p0 + lane][p0 + l] -= lij * S[p0 + l][p0 + j];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (fail_j >= 0) {
            if (tid == 0) atomicMin(&st->fail_index, (unsigned long long)(row0 + fail_j));
            return false;
        }
        const int q0 = p0 + kPW;
        // 2. rows below the panel: x L_pp^T = row, one thread per row
        if (tid < NB - q0) {
            const int i = q0 + tid;
            double x[kPW];
#pragma unroll
            for (int j = 0; j < kPW; ++j) {
                double v = S[i][p0 + j];
#pragma unroll
                for (int l = 0; l < j; ++l) v -= x[l] * S[p0 + j][p0 + l];
                x[j] = v * sm.rd[p0 + j];
            }
#pragma unroll
            for (int j = 0; j < kPW; ++j) S[i][p0 + j] = x[j];
        }
        __syncthreads();
        // 3. rank-16 update of the trailing lower triangle (rows and columns q0..NB-1)
        const int m = NB - q0;
        for (int e = tid; e < m * m; e += 256) {
            const int i = q0 + e / m, l = q0 + e % m;
            if (l <= i) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < kPW; ++j) acc = fma(S[i][p0 + j], S[l][p0 + j], acc);
                S[i][l] -= acc;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < NB * NB; e += 256) {
        const int i = e / NB, j = e % NB;
        A[(size_t)i * ld + j] = (j <= i) ? S[i][j] : 0.0;
    }
    return true;
}

__device__ __forceinline__ bool potrf64_smem_s(Potrf64Smem &sm, double *A, int ld, int64_t row0, DevStatus *st)
{
    return potrf_smem_s<64>(sm, A, ld, row0, st);
}

__device__ __forceinline__ bool potrf64_smem(double *A, int ld, int64_t row0, DevStatus *st)
{
    __shared__ Potrf64Smem sm;
    return potrf64_smem_s(sm, A, ld, row0, st);
}

// ---------------------------------------------------------------------------
// C (32 x 32, row stride ldc) -= Am (32 x K) An (32 x K)^T; 2 x 2 outputs per
// thread (rows ty + 16 i, columns tx + 16 j).  FP64 or FP32 operands, FP64
// arithmetic.  256 threads.
// ---------------------------------------------------------------------------
struct Gemm32Smem {
    double As[kPW][33];
    double Bs[kPW][33];
};

template <typename EA, typename EB>
__device__ __forceinline__ void gemm_sub32_s(Gemm32Smem &sm, const EA *Am, int lda, const EB *An, int ldb, int K,
                                             double *C, int ldc)
{
    double(&As)[kPW][33] = sm.As;
    double(&Bs)[kPW][33] = sm.Bs;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int p = 0; p < K; p += kPW) {
        for (int e = tid; e < 32 * kPW; e += 256) {
            const int r = e >> 4, l = e & 15;
            As[l][r] = (double)Am[(size_t)r * lda + p + l];
            Bs[l][r] = (double)An[(size_t)r * ldb + p + l];
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < kPW; ++l) {
            const double a0 = As[l][ty], a1 = As[l][ty + 16], b0 = Bs[l][tx], b1 = Bs[l][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) C[(size_t)(ty + 16 * i) * ldc + tx + 16 * j] -= acc[i][j];
}

template <typename EA, typename EB>
__device__ __forceinline__ void gemm_sub32(const EA *Am, int lda, const EB *An, int ldb, int K, double *C, int ldc)
{
    __shared__ Gemm32Smem sm;
    gemm_sub32_s(sm, Am, lda, An, ldb, K, C, ldc);
}

// ---------------------------------------------------------------------------
// X L^T = A for RB rows (RB in {8, 16, 64}): X and A at Xp (row stride ldx,
// ncols columns), L lower ncols x ncols at Lp (row stride ldl).  32-column
// blocks: a GEMM-style update with the already-solved columns, then a
// 32-wide substitution in shared memory.  256 threads; fewer rows per CTA put
// more SMs on a panel when the panel is short.  cstart (a multiple of 32):
// the columns before it are zero in A, hence in X, and are skipped.  TX =
// float: X and all arithmetic in FP32 (L rounded to FP32 as it is staged).
// ---------------------------------------------------------------------------
template <int RB, typename TX>
struct TrsmSmem {
    TX Xs[RB][kPW + 1];
    TX Ls[32][kPW + 1];
    TX Ab[RB][33];
    TX Ld[32][33];
};

template <int RB, typename TX = double>
__device__ __forceinline__ void trsm_rows_s(TrsmSmem<RB, TX> &sm, const double *Lp, int ldl, TX *Xp, int ldx,
                                            int ncols, int cstart = 0)
{
    constexpr int RPG = RB / 8;  // rows per thread group (8 groups of 32 threads)
    TX(&Xs)[RB][kPW + 1] = sm.Xs;
    TX(&Ls)[32][kPW + 1] = sm.Ls;
    TX(&Ab)[RB][33] = sm.Ab;
    TX(&Ld)[32][33] = sm.Ld;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    for (int c0 = cstart; c0 < ncols; c0 += 32) {
        TX acc[RPG];
#pragma unroll
        for (int i = 0; i < RPG; ++i) acc[i] = Xp[(size_t)(ty * RPG + i) * ldx + c0 + tx];
        for (int p = cstart; p < c0; p += kPW) {
            for (int e = tid; e < RB * kPW; e += 256) {
                const int r = e >> 4, l = e & 15;
                Xs[r][l] = Xp[(size_t)r * ldx + p + l];
            }
            for (int e = tid; e < 32 * kPW; e += 256) {
                const int c = e >> 4, l = e & 15;
                Ls[c][l] = (TX)Lp[(size_t)(c0 + c) * ldl + p + l];
            }
            __syncthreads();
#pragma unroll
            for (int l = 0; l < kPW; ++l) {
                const TX lv = Ls[tx][l];
#pragma unroll
                for (int i = 0; i < RPG; ++i) acc[i] = fma(-Xs[ty * RPG + i][l], lv, acc[i]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < RPG; ++i) Ab[ty * RPG + i][tx] = acc[i];
        for (int e = tid; e < 32 * 32; e += 256) {
            const int r = e >> 5, c = e & 31;
            Ld[r][c] = (c <= r) ? (TX)Lp[(size_t)(c0 + r) * ldl + c0 + c] : (TX)0;
        }
        __syncthreads();
        if (tid < RB) {
            for (int j = 0; j < 32; ++j) {
                TX s = Ab[tid][j];
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

template <int RB, typename TX = double>
__device__ __forceinline__ void trsm_rows(const double *Lp, int ldl, TX *Xp, int ldx, int ncols, int cstart = 0)
{
    __shared__ TrsmSmem<RB, TX> sm;
    trsm_rows_s<RB, TX>(sm, Lp, ldl, Xp, ldx, ncols, cstart);
}

// ---------------------------------------------------------------------------
// X L^T = A for one 32 x 32 block (the TRSM tasks of the diagonal-tile task
// graphs): X and A at Xp (row stride ldx, solved in place), L lower at Lp
// (row stride ldl).  Four threads per row split each dot product over the
// solved columns (l = q mod 4) and combine it with two shuffles in a fixed
// order, so 4 warps (one per SM sub-partition) share the substitution and
// the row's chain per column is about j / 4 FMAs, two additions and a
// multiplication by 1 / L_jj.  256 threads (warps 4-7 only stage the block).
// ---------------------------------------------------------------------------
struct Trsm32Smem {
    double X[32][33];
    double L[32][33];
    double rd[32];
};

__device__ __forceinline__ void trsm32_s(Trsm32Smem &sm, const double *Lp, int ldl, double *Xp, int ldx)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * 32; e += 256) {
        const int r = e >> 5, c = e & 31;
        sm.X[r][c] = Xp[(size_t)r * ldx + c];
        sm.L[r][c] = c <= r ? Lp[(size_t)r * ldl + c] : 0.0;
    }
    if (tid < 32) sm.rd[tid] = 1.0 / Lp[(size_t)tid * ldl + tid];
    __syncthreads();
    if (tid < 128) {
        const int r = tid >> 2, q = tid & 3;
        for (int j = 0; j < 32; ++j) {
            double part = 0.0;
            for (int l = q; l < j; l += 4) part = fma(sm.X[r][l], sm.L[j][l], part);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            const double x = (sm.X[r][j] - part) * sm.rd[j];
            __syncwarp();
            if (q == 0) sm.X[r][j] = x;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += 256) Xp[(size_t)(e >> 5) * ldx + (e & 31)] = sm.X[e >> 5][e & 31];
    __syncthreads();  // sm is free for the next block
}

// ---------------------------------------------------------------------------
// C (64 x 64, row stride ldc) -= Am (64 x K) An (64 x K)^T with row strides
// lda, ldb; the operands may be FP64 or FP32 and are converted to the
// accumulation type TC on staging (TC = double: FP64 products and sums of
// FP64 or FP32 operands; TC = float: an FP32 update of an FP32 tile).  4 x 4 outputs per thread (rows ty + 16 i, columns tx + 16 j, so a
// half-warp touches 128 contiguous bytes).  256 threads.
// ---------------------------------------------------------------------------
// Staging buffers of gemm_sub64, one set per accumulation type in a kernel
// (however many operand-type combinations it instantiates).
template <typename TC>
struct GemmSmem {
    TC As[kPW][65];
    TC Bs[kPW][65];
};
template <typename TC>
__device__ __forceinline__ GemmSmem<TC> &gemm_smem()
{
    __shared__ GemmSmem<TC> sm;
    return sm;
}

template <typename EA, typename EB, typename TC = double>
__device__ __forceinline__ void gemm_sub64_s(GemmSmem<TC> &sm, const EA *Am, int lda, const EB *An, int ldb, int K,
                                             TC *C, int ldc)
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    TC acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (TC)0;
    for (int p = 0; p < K; p += kPW) {
        for (int e = tid; e < 64 * kPW; e += 256) {
            const int r = e >> 4, l = e & 15;
            sm.As[l][r] = (TC)Am[(size_t)r * lda + p + l];
            sm.Bs[l][r] = (TC)An[(size_t)r * ldb + p + l];
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < kPW; ++l) {
            TC a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sm.As[l][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = sm.Bs[l][tx + 16 * j];
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

template <typename EA, typename EB, typename TC = double>
__device__ __forceinline__ void gemm_sub64(const EA *Am, int lda, const EB *An, int ldb, int K, TC *C, int ldc)
{
    gemm_sub64_s<EA, EB, TC>(gemm_smem<TC>(), Am, lda, An, ldb, K, C, ldc);
}

// Fixed-order tree reduction of one value per thread (any blockDim.x <= 1024).
// Returns the total (valid in every thread after the last barrier).
__device__ __forceinline__ double block_sum(double v, double *red)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    red[tid] = v;
    __syncthreads();
    int p2 = 1;
    while (p2 < nt) p2 <<= 1;
    for (int s = p2 >> 1; s > 0; s >>= 1) {
        if (tid < s && tid + s < nt) red[tid] += red[tid + s];
        __syncthreads();
    }
    return red[0];
}

// Forward substitution on one diagonal tile: y = L^-1 r in place on v
// (b entries), blockDim.x = b threads (thread i owns row i).  32-column
// blocks: the owning warp solves its 32 x 32 block with shuffles, then every
// later row subtracts the block's contribution (32 consecutive entries of its
// own row of L).  If ld_q is not NULL, ld_q[0] = sum_i log L_ii and
// ld_q[1] = sum_i y_i^2 (fixed-order trees).
__device__ __forceinline__ void trsv_fwd_tile(const double *__restrict__ L, int b, double *__restrict__ v,
                                              double *ld_q)
{
    __shared__ double yv[1024];
    __shared__ double red[1024];
    __shared__ double D[32][33];
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const double *Li = L + (size_t)i * b;
    double r = v[i];
    for (int cb = 0; cb < b / 32; ++cb) {
        const int c0 = cb * 32;
        // stage the 32 x 32 diagonal block so the warp's serial solve reads
        // shared memory instead of global memory
        for (int e = i; e < 32 * 32; e += b) D[e >> 5][e & 31] = L[(size_t)(c0 + (e >> 5)) * b + c0 + (e & 31)];
        __syncthreads();
        if (w == cb) {
            for (int jj = 0; jj < 32; ++jj) {
                const double yj = __shfl_sync(0xffffffffu, r, jj) / D[jj][jj];
                if (lane == jj) yv[c0 + jj] = yj;
                if (lane > jj) r = fma(-D[lane][jj], yj, r);
            }
        }
        __syncthreads();
        if (i >= c0 + 32) {
            double s = 0.0;
#pragma unroll 8
            for (int jj = 0; jj < 32; ++jj) s = fma(Li[c0 + jj], yv[c0 + jj], s);
            r -= s;
        }
    }
    __syncthreads();
    const double y = yv[i];
    v[i] = y;
    if (ld_q) {
        const double ld = block_sum(log(Li[i]), red);
        __syncthreads();
        const double q = block_sum(y * y, red);
        if (i == 0) {
            ld_q[0] = ld;
            ld_q[1] = q;
        }
    }
}

// z_m[r] -= L_mk[r][:] . y for the 64 rows r0..r0+63 of one panel tile, one
// warp per 8 rows with a fixed shuffle tree.  ys: the b entries of y in
// shared memory.  256 threads.
template <typename E>
__device__ __forceinline__ void gemv_rows(const E *__restrict__ A, int b, int r0, const double *ys,
                                          double *__restrict__ out)
{
    // the warp's 8 rows are swept together (8 loads in flight per lane); each
    // row's sum keeps its order, so results equal a row-by-row sweep
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const E *rows = A + (size_t)(r0 + warp * 8) * b;
    double s[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) s[rr] = 0.0;
    for (int c = lane; c < b; c += 32) {
        const double y = ys[c];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) s[rr] = fma((double)rows[(size_t)rr * b + c], y, s[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
        double v = s[rr];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) out[r0 + warp * 8 + rr] -= v;
    }
}

// Backward substitution on one diagonal tile: L^T x = r in place on v (b
// entries), blockDim.x = b (thread i owns row i).  32-column blocks from the
// last: the owning warp solves its 32 x 32 block with shuffles, then every
// thread with a smaller row index subtracts the block's contribution (L read
// along its rows).
__device__ __forceinline__ void trsv_bwd_tile(const double *__restrict__ L, int b, double *__restrict__ v)
{
    __shared__ double xv[1024];
    __shared__ double D[32][33];
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    double r = v[i];
    for (int cb = b / 32 - 1; cb >= 0; --cb) {
        const int c0 = cb * 32;
        for (int e = i; e < 32 * 32; e += b) D[e >> 5][e & 31] = L[(size_t)(c0 + (e >> 5)) * b + c0 + (e & 31)];
        __syncthreads();
        if (w == cb) {
            for (int jj = 31; jj >= 0; --jj) {
                const double xj = __shfl_sync(0xffffffffu, r, jj) / D[jj][jj];
                if (lane == jj) xv[c0 + jj] = xj;
                if (lane < jj) r = fma(-D[jj][lane], xj, r);
            }
        }
        __syncthreads();
        if (i < c0) {
            double s = 0.0;
#pragma unroll 8
            for (int jj = 0; jj < 32; ++jj) s = fma(L[(size_t)(c0 + jj) * b + i], xv[c0 + jj], s);
            r -= s;
        }
    }
    __syncthreads();
    v[i] = xv[i];
}

__device__ __forceinline__ double col_dot(const double *__restrict__ A, int b, int c, int g, const double *xs,
                                          const float *)
{
    // eight independent partial sums (rows g + 4 u mod 32) keep eight loads
    // in flight; they are combined in a fixed order
    double s[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] = 0.0;
    for (int r = g; r < b; r += 32) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] = fma(A[(size_t)(r + 4 * u) * b + c], xs[r + 4 * u], s[u]);
    }
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// Off-band (FP32) tiles: products and the partial sum in FP32 (the tile is
// only FP32 accurate; the refinement recovers the quadratic form in FP64).
__device__ __forceinline__ double col_dot(const float *__restrict__ A, int b, int c, int g, const double *,
                                          const float *xs32)
{
    float s[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] = 0.0f;
    for (int r = g; r < b; r += 32) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] = fmaf(A[(size_t)(r + 4 * u) * b + c], xs32[r + 4 * u], s[u]);
    }
    return (double)(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])));
}

// vj[c0 .. c0+63] -= (L_kj^T xk)[c0 .. c0+63] for one tile (FP64 or FP32):
// 64 columns x 4 row groups, reduced in a fixed order.  256 threads.
__device__ __forceinline__ void gemv_T_cols(const Tiles &tl, int k, int j, int c0, const double *xk, double *vj)
{
    __shared__ double xs[1024];
    __shared__ float xs32[1024];
    __shared__ double red[4][64];
    const int b = tl.b;
    const int tx = threadIdx.x & 63, g = threadIdx.x >> 6;
    for (int c = threadIdx.x; c < b; c += 256) {
        xs[c] = xk[c];
        xs32[c] = (float)xs[c];
    }
    __syncthreads();
    const double s = tl.is64(k, j) ? col_dot(tl.t64(k, j), b, c0 + tx, g, xs, xs32)
                                   : col_dot(tl.t32(k, j), b, c0 + tx, g, xs, xs32);
    red[g][tx] = s;
    __syncthreads();
    if (g == 0) vj[c0 + tx] -= ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
}

// FP32 variant for the off-band tiles of the mixed-precision solves: the
// products and the row sum run in FP32 (the tile itself is only FP32
// accurate, and the quadratic form is recovered by the FP64 refinement); the
// FP32 row sum is subtracted from the FP64 residual.  ys32: y in FP32.
__device__ __forceinline__ void gemv_rows_f32(const float *__restrict__ A, int b, int r0, const float *ys32,
                                              double *__restrict__ out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *rows = A + (size_t)(r0 + warp * 8) * b;
    float s[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) s[rr] = 0.0f;
    for (int c = lane; c < b; c += 32) {
        const float y = ys32[c];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) s[rr] = fmaf(rows[(size_t)rr * b + c], y, s[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
        float v = s[rr];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) out[r0 + warp * 8 + rr] -= (double)v;
    }
}

}  // namespace egs
