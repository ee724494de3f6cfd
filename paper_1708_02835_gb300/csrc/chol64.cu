// FP64 tile Cholesky (Algorithm 2, dpotrf) by the right-looking tile algorithm
// of Section 5.2: for k = 0..T-1
//   POTRF  L_kk = chol(A_kk)
//   TRSM   A_mk <- A_mk L_kk^-T            (m > k)
//   SYRK   A_mm <- A_mm - A_mk A_mk^T       (m > k)
//   GEMM   A_mn <- A_mn - A_mk A_nk^T       (m > n > k)
// SYRK and GEMM share one kernel (a diagonal output tile skips its upper
// sub-blocks).
//
// The diagonal POTRF is itself blocked: one launch runs the task graph of the
// tile's 32 x 32 blocks on a few dozen CTAs, so that the factorisation's
// critical path uses many SMs instead of one.
//
// GB300's FP64 rate is 2 DFMA per clock per SM (about 1.2 TFLOP/s for the
// chip), so these kernels are FP64-pipe bound whatever their memory traffic:
// the design goal is to keep every SM's FP64 pipe busy, not to save bytes.
// Every output element is updated by exactly one thread in a fixed order, so
// results are bitwise reproducible.
#include "blocks.cuh"

namespace egs {

// ---- kernels --------------------------------------------------------------

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

// ---- the diagonal-tile POTRF as one launch --------------------------------
//
// POTRF of diagonal tile k is a task graph on the nb x nb grid of its
// 32 x 32 blocks (nb = b / 32):
//   POTRF(p)       block (p, p), after its p updates; zeroes row block p right of it
//   TRSM(m, p)     block (m, p) against L_pp, after POTRF(p) and its p updates
//   UPDATE(m,n,p)  block (m, n) -= (m, p) (n, p)^T, after TRSM(m, p), TRSM(n, p)
//                  and updates 0 .. p-1 of (m, n)
// One launch of a few dozen CTAs runs it: each CTA claims the next task in
// this (topological) order from a counter and waits -- bounded, 2 s -- until
// the block counters it needs reach their values (block (i, j) counts one
// per update applied and one when final).  With 32-wide blocks the critical
// path of a sub-panel (POTRF, one 32-row solve, one 32 x 32 x 32 update) is
// short, and the many updates of early sub-panels spread over the CTAs.  The
// 32 x 32 updates of diagonal blocks also write their upper halves, which
// POTRF of the block overwrites with zeros.  The persistent batch runs the
// same block operations in the same order per element (batched_dag.cu), so
// batched and single factors agree bit for bit.  An expired wait sets
// st->timeout and stops the factorisation (reported as EGS_ERR_TIMEOUT).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool diag_wait(const unsigned *c, unsigned target, DevStatus *st)
{
    if (ld_acquire_u32(c) >= target) return true;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        __nanosleep(32);
        if (ld_acquire_u32(c) >= target) return true;
        if (failed(st)) return false;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) {
            atomicExch(&st->timeout, 1);
            atomicMin(&st->fail_index, 0ull);  // stops the rest of the evaluation
            return false;
        }
    }
}

union DiagSmem {
    PotrfSmem<32> potrf;
    Trsm32Smem trsm;
    Gemm32Smem gemm;
};

// Task t of the graph: type 0 POTRF(p), 1 TRSM(m, p), 2 UPDATE(m, n, p).
__device__ __forceinline__ void diag_decode(int t, int nb, int &type, int &p, int &m, int &n)
{
    for (p = 0; p < nb; ++p) {
        const int r = nb - p - 1, cnt = 1 + r + r * (r + 1) / 2;
        if (t < cnt) break;
        t -= cnt;
    }
    const int r = nb - p - 1;
    if (t == 0) {
        type = 0;
        m = n = p;
    } else if (t <= r) {
        type = 1;
        m = p + t;
        n = p;
    } else {
        type = 2;
        int u = t - 1 - r;
        m = p + 1;
        while (u >= m - p) {
            u -= m - p;
            ++m;
        }
        n = p + 1 + u;
    }
}

__global__ void __launch_bounds__(256) k_potrf_tile_dag(Tiles tl, int k, unsigned *ctr, DevStatus *st)
{
    __shared__ DiagSmem sm;
    __shared__ int s_task, s_ok;
    const int b = tl.b, nb = b >> 5, tid = threadIdx.x;
    int ntasks = 0;
    for (int p = 0; p < nb; ++p) {
        const int r = nb - p - 1;
        ntasks += 1 + r + r * (r + 1) / 2;
    }
    double *A = tl.t64(k, k);
    unsigned *cnt = ctr;  // block (i, j) at i (i + 1) / 2 + j
    unsigned *next = ctr + nb * (nb + 1) / 2;
    for (;;) {
        if (tid == 0) s_task = failed(st) ? ntasks : (int)atomicAdd(next, 1u);
        __syncthreads();
        const int t = s_task;
        if (t >= ntasks) return;
        int type, p, m, n;
        diag_decode(t, nb, type, p, m, n);
        if (tid == 0) {
            bool ok;
            if (type == 0) ok = diag_wait(cnt + tile_linear(p, p), (unsigned)p, st);
            else if (type == 1)
                ok = diag_wait(cnt + tile_linear(p, p), (unsigned)p + 1, st) &&
                     diag_wait(cnt + tile_linear(m, p), (unsigned)p, st);
            else
                ok = diag_wait(cnt + tile_linear(m, p), (unsigned)p + 1, st) &&
                     diag_wait(cnt + tile_linear(n, p), (unsigned)p + 1, st) &&
                     diag_wait(cnt + tile_linear(m, n), (unsigned)p, st);
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;
        double *Bmp = A + (size_t)m * 32 * b + p * 32;
        if (type == 0) {
            if (!potrf_smem_s<32>(sm.potrf, Bmp, b, (int64_t)k * b + p * 32, st)) return;
            for (int e = tid; e < 32 * (b - p * 32 - 32); e += 256) {
                const int r = e / (b - p * 32 - 32), c = e % (b - p * 32 - 32);
                Bmp[(size_t)r * b + 32 + c] = 0.0;
            }
        } else if (type == 1) {
            trsm32_s(sm.trsm, A + (size_t)p * 32 * b + p * 32, b, Bmp, b);
        } else {
            gemm_sub32_s(sm.gemm, Bmp, b, A + (size_t)n * 32 * b + p * 32, b, 32, A + (size_t)m * 32 * b + n * 32, b);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(cnt + tile_linear(m, type == 2 ? n : p), 1u);
        }
    }
}

size_t potrf_diag_scratch_words(int b)
{
    const int nb = b / 32;
    return (size_t)nb * (nb + 1) / 2 + 1;
}

cudaError_t launch_potrf_diag(const Tiles &tl, int k, DevStatus *st, cudaStream_t s, KernelTimer *kt, unsigned *ctr)
{
    // ctr: this tile's zeroed counters (potrf_diag_scratch_words(b) words)
    const int nb = tl.b / 32;
    const int grid = nb * (nb - 1) / 2 < 48 ? (nb * (nb - 1) / 2 > 1 ? nb * (nb - 1) / 2 : 1) : 48;
    EGS_LAUNCH(kt, KC_POTRF, s, k_potrf_tile_dag<<<grid, 256, 0, s>>>(tl, k, ctr, st));
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

cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s, KernelTimer *kt,
                                   unsigned *ctr)
{
    const int T = g.T;
    const Tiles tl{tiles, nullptr, g.b, T, T};
    cudaError_t e0 = cudaMemsetAsync(ctr, 0, (size_t)T * potrf_diag_scratch_words(g.b) * sizeof(unsigned), s);
    if (e0 != cudaSuccess) return e0;
    for (int k = 0; k < T; ++k) {
        if (kt) kt->step = k;
        cudaError_t e = launch_potrf_diag(tl, k, st, s, kt, ctr + (size_t)k * potrf_diag_scratch_words(g.b));
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
