// Batched evaluation of many independent likelihood problems (uneven n, own
// theta each) in FP64, or in the FP32 mixed mode (FP64 band of 2 tiles, FP32
// off-band tiles and FP32 off-band updates on the CUDA cores, FP64 updates
// of every band tile, one FP64 refinement step against an FP64 copy of
// Sigma, as in the single-problem FP32 mode): the same tile algorithm as the single-problem path
// (Algorithm 2 with the tile Cholesky of Section 5.2), but every kernel
// launch covers one step of *all* problems at once.  A launch's work items
// are the concatenation of every problem's items for that step; the CTA finds
// its problem by binary search in a per-launch prefix table, so a batch of
// 512 problems with tiles of 128 needs a few hundred launches in total, and
// the whole sequence is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "batched.cuh"
#include "batched_dag.cuh"
#include "blocks.cuh"
#include "matern.cuh"

namespace egs {

struct BatchArgs {
    const BatchProblem *probs;
    const int64_t *prefix;  // nprob + 1 item offsets for this launch
    int nprob, b;
};

// Largest p with prefix[p] <= bid (that problem owns item bid).
__device__ __forceinline__ int find_problem(const BatchArgs &a, int64_t bid, int64_t &local)
{
    int lo = 0, hi = a.nprob;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.prefix[mid] <= bid) lo = mid;
        else hi = mid;
    }
    local = bid - a.prefix[lo];
    return lo;
}

__device__ __forceinline__ Tiles dense_tiles(const BatchProblem &p, int b) { return Tiles{p.tiles, p.f32, b, p.T, p.band}; }

// Vector `which` of a problem: 0 = zpad (Z / forward solution), 1 = x, 2 = d.
__device__ __forceinline__ double *bvec(const BatchProblem &p, int which)
{
    return which == 0 ? p.zpad : (which == 1 ? p.x : p.d);
}

__device__ __forceinline__ int band_rows(const BatchProblem &p, int k)
{
    const int r = p.T - k - 1;
    return p.band - 1 < r ? p.band - 1 : r;
}

// Local polynomials of the general-nu problems (blockIdx.y = problem).
__global__ void __launch_bounds__(256) kb_table(const BatchProblem *probs)
{
    const BatchProblem &pr = probs[blockIdx.y];
    __shared__ egs_matern_params Ps;
    __shared__ double vals[8][EGS_MT_NC];
    const double *s = reinterpret_cast<const double *>(pr.P);
    double *d = reinterpret_cast<double *>(&Ps);
    for (int i = threadIdx.x; i < (int)(sizeof(egs_matern_params) / sizeof(double)); i += blockDim.x) d[i] = s[i];
    __syncthreads();
    if (Ps.kind != EGS_MATERN_GENERAL) return;
    const int w = threadIdx.x >> 5, iv = (int)blockIdx.x * 8 + w;
    if (iv < EGS_MT_OCT * EGS_MT_SUB) matern_table_interval(&Ps, iv, pr.mtab, vals[w]);
}

cudaError_t launch_batch_tables(const BatchProblem *probs, int nprob, cudaStream_t s)
{
    kb_table<<<dim3((EGS_MT_OCT * EGS_MT_SUB + 7) / 8, (unsigned)nprob), 256, 0, s>>>(probs);
    return cudaGetLastError();
}

// Matern tiles: item = (tile, 64 x 64 sub-block).
__global__ void __launch_bounds__(256) kb_gen(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    __shared__ egs_matern_params Ps;
    __shared__ double Ts[EGS_MT_DOUBLES];
    {
        const double *s = reinterpret_cast<const double *>(pr.P);
        double *d = reinterpret_cast<double *>(&Ps);
        for (int i = threadIdx.x; i < (int)(sizeof(egs_matern_params) / sizeof(double)); i += blockDim.x) d[i] = s[i];
        __syncthreads();
    }
    const bool general = Ps.kind == EGS_MATERN_GENERAL;
    if (general) {
        for (int i = threadIdx.x; i < EGS_MT_DOUBLES; i += blockDim.x) Ts[i] = pr.mtab[i];
        __syncthreads();
    }
    const double *Tab = general ? Ts : nullptr;
    const int b = a.b, nsub = b >> 6;
    const int64_t t = local / (nsub * nsub);
    const int sub = (int)(local % (nsub * nsub));
    int ti, tj;
    tri_decode(t, ti, tj);
    const int sr = sub / nsub, sc = sub % nsub;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int64_t n = pr.n;
    const int64_t gj = (int64_t)tj * b + sc * 64 + tx;
    const double xj = gj < n ? pr.X[gj] : 0.0, yj = gj < n ? pr.Y[gj] : 0.0;
    const Tiles tl = dense_tiles(pr, b);
    const bool is64 = tl.is64(ti, tj);
    double *tile = is64 ? tl.t64(ti, tj) : nullptr;
    float *tile32 = is64 ? nullptr : tl.t32(ti, tj);
    double *tsig = pr.sig ? pr.sig + (size_t)t * b * b : nullptr;
    for (int rr = 0; rr < 16; ++rr) {
        const int r = sr * 64 + ty + 4 * rr;
        const int64_t gi = (int64_t)ti * b + r;
        double v;
        if (gi >= n || gj >= n) v = (gi == gj) ? 1.0 : 0.0;
        else if (gi == gj) v = Ps.th1;
        else {
            v = matern_eval(&Ps, loc_dist(&Ps, pr.X[gi], pr.Y[gi], xj, yj) * Ps.inv_th2, Tab);
        }
        const size_t off = (size_t)r * b + sc * 64 + tx;
        if (is64) tile[off] = v;
        else tile32[off] = (float)v;
        if (tsig) tsig[off] = v;
    }
}

__global__ void __launch_bounds__(256) kb_potrf_sub(BatchArgs a, int k, int p)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b;
    double *A = dense_tiles(pr, b).t64(k, k) + (size_t)p * b + p;
    if (!potrf64_smem(A, b, (int64_t)k * b + p, pr.st)) return;
    for (int e = threadIdx.x; e < kIB * (b - p - kIB); e += 256) {
        const int r = e / (b - p - kIB), c = e % (b - p - kIB);
        A[(size_t)r * b + kIB + c] = 0.0;
    }
}

__global__ void __launch_bounds__(256) kb_trsm_sub(BatchArgs a, int k, int p)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b;
    double *A = dense_tiles(pr, b).t64(k, k);
    const int r0 = p + kIB + 16 * (int)local;
    trsm_rows<16>(A + (size_t)p * b + p, b, A + (size_t)r0 * b + p, b, kIB);
}

__global__ void __launch_bounds__(256) kb_syrk_sub(BatchArgs a, int k, int p)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b;
    double *A = dense_tiles(pr, b).t64(k, k);
    int bi, bj;
    tri_decode(local, bi, bj);
    const int q = p + kIB;
    const int ri = q + 32 * bi, rj = q + 32 * bj;
    gemm_sub32(A + (size_t)ri * b + p, b, A + (size_t)rj * b + p, b, kIB, A + (size_t)ri * b + rj, b);
}

__global__ void __launch_bounds__(256) kb_trsm_panel(BatchArgs a, int k)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b, per = b / 64;
    const Tiles tl = dense_tiles(pr, b);
    const int m = k + 1 + (int)(local / per);
    const int r0 = (int)(local % per) * 64;
    trsm_rows<64>(tl.t64(k, k), b, tl.t64(m, k) + (size_t)r0 * b, b, b);
}

// Mixed problems: the off-band rows m = k + band .. T - 1 in FP32 (L_kk
// rounded to FP32 as it is staged).
__global__ void __launch_bounds__(256) kb_trsm_panel32(BatchArgs a, int k)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b, per = b / 64;
    const Tiles tl = dense_tiles(pr, b);
    const int m = k + 1 + band_rows(pr, k) + (int)(local / per);
    const int r0 = (int)(local % per) * 64;
    trsm_rows<64, float>(tl.t64(k, k), b, tl.t32(m, k) + (size_t)r0 * b, b, b);
}

__global__ void __launch_bounds__(256) kb_update(BatchArgs a, int k)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b, nsub = b >> 6;
    const Tiles tl = dense_tiles(pr, b);
    int mm, nn;
    tri_decode(local / (nsub * nsub), mm, nn);
    const int sub = (int)(local % (nsub * nsub));
    const int m = k + 1 + mm, nc = k + 1 + nn;
    const int sr = sub / nsub, sc = sub % nsub;
    if (m == nc && sc > sr) return;
    const size_t ao = (size_t)sr * 64 * b, bo = (size_t)sc * 64 * b, co = (size_t)sr * 64 * b + sc * 64;
    if (tl.is64(m, nc)) {
        // band (or FP64) output: FP64 products of the stored operands
        if (tl.is64(m, k)) {
            if (tl.is64(nc, k)) gemm_sub64(tl.t64(m, k) + ao, b, tl.t64(nc, k) + bo, b, b, tl.t64(m, nc) + co, b);
            else gemm_sub64(tl.t64(m, k) + ao, b, tl.t32(nc, k) + bo, b, b, tl.t64(m, nc) + co, b);
        } else {
            if (tl.is64(nc, k)) gemm_sub64(tl.t32(m, k) + ao, b, tl.t64(nc, k) + bo, b, b, tl.t64(m, nc) + co, b);
            else gemm_sub64(tl.t32(m, k) + ao, b, tl.t32(nc, k) + bo, b, b, tl.t64(m, nc) + co, b);
        }
    } else {
        // off-band output (then m - k > band, so A_mk is FP32): FP32 update
        if (tl.is64(nc, k)) gemm_sub64(tl.t32(m, k) + ao, b, tl.t64(nc, k) + bo, b, b, tl.t32(m, nc) + co, b);
        else gemm_sub64(tl.t32(m, k) + ao, b, tl.t32(nc, k) + bo, b, b, tl.t32(m, nc) + co, b);
    }
}

__global__ void kb_pad(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    const int64_t i = local * 256 + threadIdx.x;
    if (i < (int64_t)pr.T * a.b) pr.zpad[i] = i < pr.n ? pr.z[i] : 0.0;
}

__global__ void __launch_bounds__(1024) kb_trsv_diag(BatchArgs a, int k, int which)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    __shared__ double ldq[2];
    trsv_fwd_tile(dense_tiles(pr, a.b).t64(k, k), a.b, bvec(pr, which) + (size_t)k * a.b, which == 0 ? ldq : nullptr);
    if (which == 0 && threadIdx.x == 0) {
        pr.partials[k] = ldq[0];
        pr.partials[pr.T + k] = ldq[1];
    }
}

__global__ void __launch_bounds__(256) kb_gemv_panel(BatchArgs a, int k, int which)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    extern __shared__ double ys[];
    const int b = a.b, per = b / 64;
    const int m = k + 1 + (int)(local / per);
    const int r0 = (int)(local % per) * 64;
    double *v = bvec(pr, which);
    float *ys32 = reinterpret_cast<float *>(ys + b);
    for (int c = threadIdx.x; c < b; c += 256) {
        ys[c] = v[(size_t)k * b + c];
        ys32[c] = (float)ys[c];
    }
    __syncthreads();
    const Tiles tl = dense_tiles(pr, b);
    if (tl.is64(m, k)) gemv_rows(tl.t64(m, k), b, r0, ys, v + (size_t)m * b);
    else gemv_rows_f32(tl.t32(m, k), b, r0, ys32, v + (size_t)m * b);
}

// ---- mixed problems: backward solves, the FP64 refinement and l ----------

// dst = src over the T*b entries (item = 256 entries).
__global__ void kb_copy(BatchArgs a, int dst, int src)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int64_t i = local * 256 + threadIdx.x;
    if (i < (int64_t)pr.T * a.b) bvec(pr, dst)[i] = bvec(pr, src)[i];
}

__global__ void __launch_bounds__(1024) kb_trsv_diag_T(BatchArgs a, int k, int which)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st) || k >= pr.T) return;
    trsv_bwd_tile(dense_tiles(pr, a.b).t64(k, k), a.b, bvec(pr, which) + (size_t)k * a.b);
}

// r_j -= L_kj^T x_k, item = (j < k, 64-column block).
__global__ void __launch_bounds__(256) kb_gemv_T(BatchArgs a, int k, int which)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b, per = b / 64;
    const int j = (int)(local / per), c0 = (int)(local % per) * 64;
    double *v = bvec(pr, which);
    gemv_T_cols(dense_tiles(pr, b), k, j, c0, v + (size_t)k * b, v + (size_t)j * b);
}

// rows[i b + r] = sum_{j <= i} Sigma_ij[r][:] . x_j; item = (i, 8 rows).
__global__ void __launch_bounds__(256) kb_symv_rows(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int b = a.b, per = b / 8;
    const int i = (int)(local / per), lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (int)(local % per) * 8 + warp;
    const size_t bb = (size_t)b * b;
    double s = 0.0;
    for (int j = 0; j <= i; ++j) {
        const double *row = pr.sig + (size_t)tile_linear(i, j) * bb + (size_t)r * b;
        const double *xj = pr.x + (size_t)j * b;
        for (int c = lane; c < b; c += 32) s = fma(row[c], xj[c], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) pr.rows[(size_t)i * b + r] = s;
}

// cols[i b + c] = sum_{m > i} Sigma_mi[:, c] . x_m; item = (i, 64 columns).
__global__ void __launch_bounds__(256) kb_symv_cols(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    __shared__ double red[4][64];
    const int b = a.b, per = b / 64;
    const int i = (int)(local / per), c0 = (int)(local % per) * 64;
    const int tx = threadIdx.x & 63, g = threadIdx.x >> 6;
    const size_t bb = (size_t)b * b;
    double s = 0.0;
    for (int m = i + 1; m < pr.T; ++m) {
        const double *A = pr.sig + (size_t)tile_linear(m, i) * bb + c0 + tx;
        const double *xm = pr.x + (size_t)m * b;
        for (int r = g; r < b; r += 4) s = fma(A[(size_t)r * b], xm[r], s);
    }
    red[g][tx] = s;
    __syncthreads();
    if (g == 0) pr.cols[(size_t)i * b + c0 + tx] = ((red[0][tx] + red[1][tx]) + red[2][tx]) + red[3][tx];
}

// d = z - (rows + cols) (z padded with zeros), item = 256 entries.
__global__ void kb_residual(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int64_t i = local * 256 + threadIdx.x;
    if (i < (int64_t)pr.T * a.b) pr.d[i] = (i < pr.n ? pr.z[i] : 0.0) - (pr.rows[i] + pr.cols[i]);
}

__global__ void kb_axpy(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    if (failed(pr.st)) return;
    const int64_t i = local * 256 + threadIdx.x;
    if (i < (int64_t)pr.T * a.b) pr.x[i] += pr.d[i];
}

// l from the log-det partials and the refined quadratic form z . x;
// result[3] keeps y . y (the unrefined one) for the accuracy check.
__global__ void __launch_bounds__(256) kb_finalize_mixed(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    __shared__ double red[256];
    double s = 0.0, q0 = 0.0, q = 0.0;
    for (int t = threadIdx.x; t < pr.T; t += 256) {
        s += pr.partials[t];
        q0 += pr.partials[pr.T + t];
    }
    for (int64_t i = threadIdx.x; i < pr.n; i += 256) q = fma(pr.z[i], pr.x[i], q);
    const double lsum = block_sum(s, red);
    __syncthreads();
    const double q0sum = block_sum(q0, red);
    __syncthreads();
    const double qsum = block_sum(q, red);
    if (threadIdx.x == 0) {
        DevStatus *st = pr.st;
        if (failed(st)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            st->result[0] = st->result[1] = st->result[2] = st->result[3] = nan;
        } else {
            const double logdet = 2.0 * lsum;
            st->result[0] = -0.5 * qsum - 0.5 * logdet - 0.5 * (double)pr.n * 1.8378770664093454836;
            st->result[1] = logdet;
            st->result[2] = qsum;
            st->result[3] = q0sum;
        }
    }
}

__global__ void __launch_bounds__(256) kb_finalize(BatchArgs a)
{
    int64_t local;
    const BatchProblem &pr = a.probs[find_problem(a, blockIdx.x, local)];
    __shared__ double red[256];
    double s = 0.0, q = 0.0;
    for (int t = threadIdx.x; t < pr.T; t += 256) {
        s += pr.partials[t];
        q += pr.partials[pr.T + t];
    }
    const double lsum = block_sum(s, red);
    __syncthreads();
    const double qsum = block_sum(q, red);
    if (threadIdx.x == 0) {
        DevStatus *st = pr.st;
        if (failed(st)) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            st->result[0] = st->result[1] = st->result[2] = nan;
        } else {
            const double logdet = 2.0 * lsum;
            st->result[0] = -0.5 * qsum - 0.5 * logdet - 0.5 * (double)pr.n * 1.8378770664093454836;
            st->result[1] = logdet;
            st->result[2] = qsum;
        }
    }
}

}  // namespace egs

// ---------------------------------------------------------------------------
// Host side: plan, graph capture and the C ABI.
// ---------------------------------------------------------------------------
using namespace egs;

struct egs_batch {
    int nprob = 0, b = 0;
    bool mixed = false;  // EGS_MIX_FP32 batch (band kBatchBand)
    int band = 0;
    std::vector<int64_t> n;
    std::vector<int> T;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Allocator alloc{};  // the allocator that provided ws
    BatchProblem *d_probs = nullptr;
    egs_matern_params *d_params = nullptr;
    DevStatus *d_status = nullptr;
    int64_t *d_prefix = nullptr;
    double *d_inputs = nullptr;  // staged locations and z (3 n per problem)
    std::vector<size_t> in_off;  // offset of problem p's inputs in d_inputs (doubles)
    BatchProblem *h_probs = nullptr;     // pinned
    egs_matern_params *h_params = nullptr;  // pinned
    DevStatus *h_status = nullptr;          // pinned
    struct Launch {
        int kind, k, p;
        size_t prefix_off;
        int64_t items;
    };
    std::vector<Launch> launches;
    cudaStream_t cs = nullptr;  // capture / replay stream
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int launches_per_run = 0;
    // persistent scheduler (FP64 batches with tile <= 256): one launch over
    // the task list of every problem
    bool dag = false;
    int4 *d_tasks = nullptr;
    long long ntasks = 0;
    unsigned *d_cnt = nullptr;
    size_t ncnt = 0;
    DagCtl *d_ctl = nullptr;
    DagCtl *h_ctl = nullptr;  // pinned: [0] written before a run, [1] read back after it
    int grid = 0;
    unsigned long long limit_ns = kDagWaitLimitNs;
    long long withhold = -1;
};

namespace {

enum {
    L_GEN, L_POTRF, L_TRSM_SUB, L_SYRK_SUB, L_TRSM, L_TRSM32, L_UPDATE, L_PAD, L_TRSV, L_GEMV, L_FINAL,
    L_COPY, L_TRSV_T, L_GEMV_T, L_SYMV_R, L_SYMV_C, L_RESID, L_AXPY, L_FINAL_M
};

constexpr int kBatchBand = 2;  // FP64 band of the mixed batches (tiles)

// Tile table of the autotuner: [ceil(log2(largest n))][precision], 0 = not tuned.
std::mutex g_tune_mu;
int32_t g_tuned[64][4] = {};

int size_class(int64_t nmax)
{
    int c = 0;
    while (c < 63 && ((int64_t)1 << c) < nmax) ++c;
    return c;
}

int32_t tuned_tile(int64_t nmax, egs_precision p)
{
    if ((int)p < 0 || (int)p > 3) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned[size_class(nmax)][(int)p];
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

void plan_launches(egs_batch *B, std::vector<int64_t> &prefix)
{
    const int b = B->b, nsub = b / 64, per = b / 64, np = B->nprob;
    int Tmax = 0;
    for (int t : B->T) Tmax = std::max(Tmax, t);
    auto add = [&](int kind, int k, int p, auto count) {
        B->launches.push_back({kind, k, p, prefix.size(), 0});
        int64_t acc = 0;
        for (int q = 0; q < np; ++q) {
            prefix.push_back(acc);
            acc += count(q);
        }
        prefix.push_back(acc);
        B->launches.back().items = acc;
    };
    auto band_of = [&](int q) { return B->mixed ? std::min(kBatchBand, B->T[q]) : B->T[q]; };
    auto nb_of = [&](int q, int k) { return (int64_t)std::min(band_of(q) - 1, B->T[q] - k - 1); };
    auto vec_items = [&](int q) { return ((int64_t)B->T[q] * b + 255) / 256; };
    add(L_GEN, 0, 0, [&](int q) { return (int64_t)B->T[q] * (B->T[q] + 1) / 2 * nsub * nsub; });
    for (int k = 0; k < Tmax; ++k) {
        for (int p = 0; p < b; p += kIB) {
            const int64_t nrest = (b - p - kIB) / 16, n32 = (b - p - kIB) / 32;
            add(L_POTRF, k, p, [&](int q) { return (int64_t)(B->T[q] > k ? 1 : 0); });
            if (nrest > 0) {
                add(L_TRSM_SUB, k, p, [&](int q) { return B->T[q] > k ? nrest : (int64_t)0; });
                add(L_SYRK_SUB, k, p, [&](int q) { return B->T[q] > k ? n32 * (n32 + 1) / 2 : (int64_t)0; });
            }
        }
        add(L_TRSM, k, 0, [&](int q) { return B->T[q] > k + 1 ? nb_of(q, k) * per : (int64_t)0; });
        if (B->mixed)
            add(L_TRSM32, k, 0, [&](int q) {
                return B->T[q] > k + 1 ? ((int64_t)(B->T[q] - k - 1) - nb_of(q, k)) * per : (int64_t)0;
            });
        add(L_UPDATE, k, 0, [&](int q) {
            const int64_t r = B->T[q] - k - 1;
            return r > 0 ? r * (r + 1) / 2 * nsub * nsub : (int64_t)0;
        });
    }
    add(L_PAD, 0, 0, vec_items);
    auto forward = [&](int which) {
        for (int k = 0; k < Tmax; ++k) {
            add(L_TRSV, k, which, [&](int q) { return (int64_t)(B->T[q] > k ? 1 : 0); });
            add(L_GEMV, k, which,
                [&](int q) { return B->T[q] > k + 1 ? (int64_t)(B->T[q] - k - 1) * per : (int64_t)0; });
        }
    };
    auto backward = [&](int which) {
        for (int k = Tmax - 1; k >= 0; --k) {
            add(L_TRSV_T, k, which, [&](int q) { return (int64_t)(B->T[q] > k ? 1 : 0); });
            if (k > 0) add(L_GEMV_T, k, which, [&](int q) { return B->T[q] > k ? (int64_t)k * per : (int64_t)0; });
        }
    };
    forward(0);  // y = L^-1 z in zpad, log-det and y.y partials
    if (!B->mixed) {
        add(L_FINAL, 0, 0, [&](int) { return (int64_t)1; });
        return;
    }
    add(L_COPY, 0, 1 * 4 + 0, vec_items);  // x = y
    backward(1);                           // x = L^-T y
    add(L_SYMV_R, 0, 0, [&](int q) { return (int64_t)B->T[q] * (b / 8); });
    add(L_SYMV_C, 0, 0, [&](int q) { return (int64_t)B->T[q] * per; });
    add(L_RESID, 0, 0, vec_items);         // d = z - Sigma x
    forward(2);
    backward(2);                           // d = L^-T L^-1 d
    add(L_AXPY, 0, 0, vec_items);          // x += d
    add(L_FINAL_M, 0, 0, [&](int) { return (int64_t)1; });
}

cudaError_t enqueue_all(egs_batch *B, cudaStream_t s)
{
    cudaError_t et = launch_batch_tables(B->d_probs, B->nprob, s);
    if (et != cudaSuccess) return et;
    if (B->dag) {
        cudaError_t e = cudaMemsetAsync(B->d_cnt, 0, B->ncnt * sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_ctl, B->h_ctl, sizeof(DagCtl), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = dag_enqueue(B->d_tasks, B->ntasks, B->d_probs, B->d_ctl, B->b, B->grid, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B->h_ctl + 1, B->d_ctl, sizeof(DagCtl), cudaMemcpyDeviceToHost, s);
        B->launches_per_run = 2;  // the local polynomials, then the persistent launch
        return e;
    }
    int count = 1;
    for (const auto &L : B->launches) {
        if (L.items <= 0) continue;
        BatchArgs a{B->d_probs, B->d_prefix + L.prefix_off, B->nprob, B->b};
        const unsigned g = (unsigned)L.items;
        switch (L.kind) {
        case L_GEN: kb_gen<<<g, 256, 0, s>>>(a); break;
        case L_POTRF: kb_potrf_sub<<<g, 256, 0, s>>>(a, L.k, L.p); break;
        case L_TRSM_SUB: kb_trsm_sub<<<g, 256, 0, s>>>(a, L.k, L.p); break;
        case L_SYRK_SUB: kb_syrk_sub<<<g, 256, 0, s>>>(a, L.k, L.p); break;
        case L_TRSM: kb_trsm_panel<<<g, 256, 0, s>>>(a, L.k); break;
        case L_TRSM32: kb_trsm_panel32<<<g, 256, 0, s>>>(a, L.k); break;
        case L_UPDATE: kb_update<<<g, 256, 0, s>>>(a, L.k); break;
        case L_PAD: kb_pad<<<g, 256, 0, s>>>(a); break;
        case L_TRSV: kb_trsv_diag<<<g, B->b, 0, s>>>(a, L.k, L.p); break;
        case L_GEMV:
            kb_gemv_panel<<<g, 256, (size_t)B->b * (sizeof(double) + sizeof(float)), s>>>(a, L.k, L.p);
            break;
        case L_FINAL: kb_finalize<<<g, 256, 0, s>>>(a); break;
        case L_COPY: kb_copy<<<g, 256, 0, s>>>(a, L.p / 4, L.p % 4); break;
        case L_TRSV_T: kb_trsv_diag_T<<<g, B->b, 0, s>>>(a, L.k, L.p); break;
        case L_GEMV_T: kb_gemv_T<<<g, 256, 0, s>>>(a, L.k, L.p); break;
        case L_SYMV_R: kb_symv_rows<<<g, 256, 0, s>>>(a); break;
        case L_SYMV_C: kb_symv_cols<<<g, 256, 0, s>>>(a); break;
        case L_RESID: kb_residual<<<g, 256, 0, s>>>(a); break;
        case L_AXPY: kb_axpy<<<g, 256, 0, s>>>(a); break;
        case L_FINAL_M: kb_finalize_mixed<<<g, 256, 0, s>>>(a); break;
        }
        ++count;
    }
    B->launches_per_run = count;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

egs_status egs_batch_create(int32_t nprob, const int64_t *n, int32_t tile, egs_precision p, egs_batch **out)
{
    if (!out || !n || nprob < 1) return set_error(EGS_ERR_ARG, "egs_batch_create: bad arguments");
    *out = nullptr;
    if (p != EGS_FP64 && p != EGS_MIX_FP32)
        return set_error(EGS_ERR_UNIMPLEMENTED, "egs_batch_create: batches are EGS_FP64 or EGS_MIX_FP32");
    if (tile == 0) {
        int64_t nmax = 0;
        for (int i = 0; i < nprob; ++i) nmax = std::max(nmax, n[i]);
        tile = tuned_tile(nmax, p);
        if (tile == 0) tile = nmax <= 2048 ? 64 : 128;
    }
    if (tile < 64 || tile > 1024 || tile % 64) return set_error(EGS_ERR_ARG, "egs_batch_create: tile %d invalid", tile);
    egs_batch *B = new egs_batch;
    B->nprob = nprob;
    B->b = tile;
    B->mixed = (p == EGS_MIX_FP32);
    size_t off = 0;
    std::vector<size_t> tiles_off(nprob), zpad_off(nprob), part_off(nprob), f32_off(nprob), sig_off(nprob),
        vec_off(nprob), mtab_off(nprob);
    size_t in_doubles = 0;
    for (int i = 0; i < nprob; ++i) {
        if (n[i] < 1) {
            delete B;
            return set_error(EGS_ERR_ARG, "egs_batch_create: n[%d] = %lld", i, (long long)n[i]);
        }
        const int T = (int)((n[i] + tile - 1) / tile);
        const int band = B->mixed ? std::min(kBatchBand, T) : T;
        const size_t bb = (size_t)tile * tile, npad = (size_t)T * tile;
        B->n.push_back(n[i]);
        B->T.push_back(T);
        tiles_off[i] = off;
        off += a256(Tiles::f64_tiles(T, band) * bb * sizeof(double));
        f32_off[i] = off;
        off += a256(Tiles::f32_tiles(T, band) * bb * sizeof(float));
        sig_off[i] = off;
        if (B->mixed) off += a256((size_t)T * (T + 1) / 2 * bb * sizeof(double));
        vec_off[i] = off;
        if (B->mixed) off += 4 * a256(npad * sizeof(double));
        zpad_off[i] = off;
        off += a256(npad * sizeof(double));
        part_off[i] = off;
        off += a256((size_t)2 * T * sizeof(double));
        mtab_off[i] = off;
        off += a256(EGS_MT_DOUBLES * sizeof(double));
        B->in_off.push_back(in_doubles);
        in_doubles += (size_t)3 * n[i];
    }
    const size_t probs_off = off;
    off += a256(sizeof(BatchProblem) * nprob);
    const size_t params_off = off;
    off += a256(sizeof(egs_matern_params) * nprob);
    const size_t status_off = off;
    off += a256(sizeof(DevStatus) * nprob);
    const size_t inputs_off = off;
    off += a256(in_doubles * sizeof(double));
    std::vector<int64_t> prefix;
    std::vector<int4> tasks;
    std::vector<size_t> cnt_off;
    B->dag = !B->mixed && tile <= 256;
    if (B->dag) {
        egs_status sc = dag_plan(B->T, tile, tasks, cnt_off, B->ncnt);
        if (sc != EGS_OK) {
            delete B;
            return sc;
        }
        B->ntasks = (long long)tasks.size();
    } else {
        plan_launches(B, prefix);
    }
    const size_t prefix_off = off;
    off += a256(prefix.size() * sizeof(int64_t));
    const size_t tasks_off = off;
    off += a256(tasks.size() * sizeof(int4));
    const size_t cnt_off_bytes = off;
    off += a256(B->ncnt * sizeof(unsigned));
    const size_t ctl_off = off;
    off += a256(sizeof(DagCtl));
    B->ws_bytes = off;
    B->alloc = current_allocator();
    cudaError_t e;
    if (!B->alloc.alloc) {
        e = cudaMalloc((void **)&B->ws, off);
    } else {  // the caller's hook, on the legacy stream (the batch outlives any call's stream)
        e = dev_alloc(B->alloc, (void **)&B->ws, off, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    }
    if (e != cudaSuccess) {
        delete B;
        return cuda_error(e, "egs_batch_create workspace");
    }
    B->d_probs = (BatchProblem *)(B->ws + probs_off);
    B->d_params = (egs_matern_params *)(B->ws + params_off);
    B->d_status = (DevStatus *)(B->ws + status_off);
    B->d_inputs = (double *)(B->ws + inputs_off);
    B->d_prefix = (int64_t *)(B->ws + prefix_off);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&B->h_probs, sizeof(BatchProblem) * nprob);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&B->h_params, sizeof(egs_matern_params) * nprob);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&B->h_status, sizeof(DevStatus) * nprob);
    if (e == cudaSuccess && !prefix.empty())
        e = cudaMemcpy(B->d_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (B->dag) {
        B->d_tasks = (int4 *)(B->ws + tasks_off);
        B->d_cnt = (unsigned *)(B->ws + cnt_off_bytes);
        B->d_ctl = (DagCtl *)(B->ws + ctl_off);
        B->grid = dag_grid();
        if (B->grid < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = cudaMallocHost((void **)&B->h_ctl, 2 * sizeof(DagCtl));
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        egs_batch_destroy(B);
        return cuda_error(e, "egs_batch_create");
    }
    for (int i = 0; i < nprob; ++i) {
        BatchProblem &pr = B->h_probs[i];
        std::memset(&pr, 0, sizeof(pr));
        double *in = B->d_inputs + B->in_off[i];
        pr.X = in;
        pr.Y = in + n[i];
        pr.z = in + 2 * n[i];
        pr.n = n[i];
        pr.T = B->T[i];
        pr.band = B->mixed ? std::min(kBatchBand, pr.T) : pr.T;
        pr.tiles = (double *)(B->ws + tiles_off[i]);
        if (B->mixed) {
            const size_t vstride = a256((size_t)pr.T * tile * sizeof(double));
            char *v = B->ws + vec_off[i];
            pr.f32 = (float *)(B->ws + f32_off[i]);
            pr.sig = (double *)(B->ws + sig_off[i]);
            pr.x = (double *)v;
            pr.d = (double *)(v + vstride);
            pr.rows = (double *)(v + 2 * vstride);
            pr.cols = (double *)(v + 3 * vstride);
        }
        pr.zpad = (double *)(B->ws + zpad_off[i]);
        pr.partials = (double *)(B->ws + part_off[i]);
        pr.st = B->d_status + i;
        pr.P = B->d_params + i;
        pr.cnt = B->dag ? B->d_cnt + cnt_off[i] : nullptr;
        pr.mtab = (double *)(B->ws + mtab_off[i]);
    }
    e = cudaMemcpy(B->d_probs, B->h_probs, sizeof(BatchProblem) * nprob, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        egs_batch_destroy(B);
        return cuda_error(e, "egs_batch_create");
    }
    *out = B;
    return EGS_OK;
}

}  // extern "C"

namespace {

// After the inputs have been staged on B->cs: the parameters, the graph
// (captured on first use) and the statuses back to the host; synchronises.
cudaError_t run_staged(egs_batch *B, cudaStream_t us, cudaError_t e)
{
    if (B->dag) {
        std::memset(B->h_ctl, 0, 2 * sizeof(DagCtl));
        B->h_ctl[0].limit_ns = B->limit_ns;
        B->h_ctl[0].withhold = B->withhold;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_params, B->h_params, sizeof(egs_matern_params) * B->nprob, cudaMemcpyHostToDevice, B->cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_status, 0xFF, sizeof(DevStatus) * B->nprob, B->cs);
    if (e == cudaSuccess && !B->exec) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_all(B, B->cs);
            e = cudaStreamEndCapture(B->cs, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->h_status, B->d_status, sizeof(DevStatus) * B->nprob, cudaMemcpyDeviceToHost, B->cs);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev_out, B->cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(us, B->ev_out, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->cs);
    return e;
}

}  // namespace

extern "C" {

egs_status egs_batch_run(egs_batch *B, const double *const *locs, const double *const *z, const double *theta,
                         double *out, egs_status *per_status, void *stream)
{
    if (!B || !locs || !z || !theta) return set_error(EGS_ERR_ARG, "egs_batch_run: NULL argument");
    cudaStream_t us = (cudaStream_t)stream;
    for (int i = 0; i < B->nprob; ++i)
        if (egs_matern_params_init(theta + 3 * i, &B->h_params[i]) != 0)
            return set_error(EGS_ERR_ARG, "egs_batch_run: theta of problem %d must be finite and > 0", i);
    cudaError_t e = cudaEventRecord(B->ev_in, us);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cs, B->ev_in, 0);
    // inputs: copied into the plan's staging area (device or host sources)
    for (int i = 0; i < B->nprob && e == cudaSuccess; ++i) {
        double *in = B->d_inputs + B->in_off[i];
        e = cudaMemcpyAsync(in, locs[i], (size_t)2 * B->n[i] * sizeof(double), cudaMemcpyDefault, B->cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(in + 2 * B->n[i], z[i], (size_t)B->n[i] * sizeof(double), cudaMemcpyDefault, B->cs);
    }
    e = run_staged(B, us, e);
    if (e != cudaSuccess) return cuda_error(e, "egs_batch_run");
    if (B->dag && B->h_ctl[1].timeouts > 0) {
        for (int i = 0; i < B->nprob; ++i) {
            if (out) out[i] = NAN;
            if (per_status) per_status[i] = EGS_ERR_TIMEOUT;
        }
        return set_error(EGS_ERR_TIMEOUT, "egs_batch_run: %u dependency wait(s) of the persistent launch ran out of "
                                          "time; the run was abandoned", B->h_ctl[1].timeouts);
    }
    egs_status worst = EGS_OK;
    for (int i = 0; i < B->nprob; ++i) {
        const DevStatus &h = B->h_status[i];
        egs_status si = EGS_OK;
        if (h.fail_index != kNoFail) si = EGS_ERR_NOT_PD;
        else if (B->mixed && std::fabs(h.result[2] - h.result[3]) > kRefineTolFp32 * std::fabs(h.result[2]))
            si = EGS_ERR_INACCURATE;
        if (out) out[i] = si == EGS_OK ? h.result[0] : NAN;
        if (per_status) per_status[i] = si;
        if (si != EGS_OK && worst != EGS_ERR_NOT_PD) worst = si;
    }
    if (worst == EGS_ERR_NOT_PD) set_error(worst, "egs_batch_run: at least one problem is not positive definite");
    else if (worst != EGS_OK) set_error(worst, "egs_batch_run: at least one mixed-precision problem is too inexact");
    return worst;
}

int32_t egs_batch_launches(const egs_batch *B) { return B ? B->launches_per_run : 0; }

int64_t egs_batch_tasks(const egs_batch *B) { return B && B->dag ? (int64_t)B->ntasks : 0; }

egs_status egs_batch_set_wait_limit(egs_batch *B, int64_t limit_ns, int64_t withhold_task)
{
    if (!B) return set_error(EGS_ERR_ARG, "egs_batch_set_wait_limit: NULL batch");
    if (!B->dag) return set_error(EGS_ERR_UNIMPLEMENTED, "egs_batch_set_wait_limit: not a persistent batch");
    if (limit_ns < 1 || withhold_task < -1 || withhold_task >= (int64_t)B->ntasks)
        return set_error(EGS_ERR_ARG, "egs_batch_set_wait_limit: limit %lld ns or task %lld out of range",
                         (long long)limit_ns, (long long)withhold_task);
    B->limit_ns = (unsigned long long)limit_ns;
    B->withhold = withhold_task;
    return EGS_OK;
}

int32_t egs_batch_tile(const egs_batch *B) { return B ? B->b : 0; }

int32_t egs_batch_tuned_tile(int64_t nmax, egs_precision p) { return nmax >= 1 ? tuned_tile(nmax, p) : 0; }

egs_status egs_batch_autotune(int32_t nprob, const int64_t *n, const double *const *locs, const double *const *z,
                              const double *theta, egs_precision p, int32_t *best_tile, double *ms, void *stream)
{
    if (!n || !locs || !z || !theta || nprob < 1) return set_error(EGS_ERR_ARG, "egs_batch_autotune: bad arguments");
    static const int32_t cand[3] = {64, 128, 256};
    cudaStream_t us = (cudaStream_t)stream;
    int32_t best = 0;
    double best_ms = 0.0;
    for (int c = 0; c < 3; ++c) {
        egs_batch *B = nullptr;
        egs_status st = egs_batch_create(nprob, n, cand[c], p, &B);
        if (st != EGS_OK) return st;
        // first run captures the graph; the second is timed
        st = egs_batch_run(B, locs, z, theta, nullptr, nullptr, stream);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float t = 0.f;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, us);
        if (e == cudaSuccess && (st == EGS_OK || st == EGS_ERR_NOT_PD || st == EGS_ERR_INACCURATE))
            st = egs_batch_run(B, locs, z, theta, nullptr, nullptr, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, us);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        egs_batch_destroy(B);
        if (e != cudaSuccess) return cuda_error(e, "egs_batch_autotune");
        if (st != EGS_OK && st != EGS_ERR_NOT_PD && st != EGS_ERR_INACCURATE) return st;
        if (ms) ms[c] = t;
        if (best == 0 || t < best_ms) {
            best = cand[c];
            best_ms = t;
        }
    }
    int64_t nmax = 0;
    for (int i = 0; i < nprob; ++i) nmax = std::max(nmax, n[i]);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[size_class(nmax)][(int)p] = best;
    }
    if (best_tile) *best_tile = best;
    clear_error();
    return EGS_OK;
}

size_t egs_batch_workspace_bytes(const egs_batch *B) { return B ? B->ws_bytes : 0; }

egs_status egs_batch_destroy(egs_batch *B)
{
    if (!B) return EGS_OK;
    if (B->cs) cudaStreamSynchronize(B->cs);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->cs) cudaStreamDestroy(B->cs);
    if (B->ws) {
        if (!B->alloc.alloc) cudaFree(B->ws);
        else dev_free(B->alloc, B->ws, B->ws_bytes, nullptr);
    }
    if (B->h_probs) cudaFreeHost(B->h_probs);
    if (B->h_params) cudaFreeHost(B->h_params);
    if (B->h_status) cudaFreeHost(B->h_status);
    if (B->h_ctl) cudaFreeHost(B->h_ctl);
    delete B;
    return EGS_OK;
}

egs_status egs_loglik_batched(int32_t nprob, const int64_t *n, const double *const *locs, const double *const *z,
                              const double *theta, egs_precision p, double *out, egs_status *per_status, void *stream)
{
    egs_batch *B = nullptr;
    egs_status st = egs_batch_create(nprob, n, 0, p, &B);
    if (st != EGS_OK) return st;
    st = egs_batch_run(B, locs, z, theta, out, per_status, stream);
    egs_batch_destroy(B);
    return st;
}


// Independent-blocks (IND) approximation (Section 6.8): every tile outside
// the diagonal super tiles of super_tiles x super_tiles tiles is set to
// zero, so Sigma is block diagonal over consecutive runs of
// super_tiles * tile locations and l_IND is the sum of Eq. 1 over the
// blocks.  The blocks are independent problems of the batched scheduler.
egs_status egs_loglik_ind(const double *locs, const double *z, const double theta[3], int64_t n, int32_t tile,
                          int32_t super_tiles, double *out_loglik, egs_info *info, void *stream)
{
    if (!locs || !z || !theta) return set_error(EGS_ERR_ARG, "egs_loglik_ind: NULL pointer");
    if (n < 1) return set_error(EGS_ERR_ARG, "egs_loglik_ind: n = %lld must be >= 1", (long long)n);
    if (super_tiles < 1) return set_error(EGS_ERR_ARG, "egs_loglik_ind: super_tiles = %d must be >= 1", super_tiles);
    if (tile == 0) tile = 128;
    if (tile < 64 || tile > 1024 || tile % 64) return set_error(EGS_ERR_ARG, "egs_loglik_ind: tile %d invalid", tile);
    egs_matern_params P;
    if (egs_matern_params_init(theta, &P) != 0) return set_error(EGS_ERR_ARG, "egs_loglik_ind: theta must be finite and > 0");
    const int64_t bs = (int64_t)super_tiles * tile;
    const int64_t nblk = (n + bs - 1) / bs;
    if (nblk > (1 << 20)) return set_error(EGS_ERR_ARG, "egs_loglik_ind: too many blocks");
    std::vector<int64_t> ns((size_t)nblk);
    for (int64_t i = 0; i < nblk; ++i) ns[(size_t)i] = std::min(bs, n - i * bs);
    egs_batch *B = nullptr;
    egs_status sc = egs_batch_create((int32_t)nblk, ns.data(), tile, EGS_FP64, &B);
    if (sc != EGS_OK) return sc;
    for (int i = 0; i < B->nprob; ++i) B->h_params[i] = P;
    cudaStream_t us = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(B->ev_in, us);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cs, B->ev_in, 0);
    // block i: x[i bs ..], y[i bs ..] (y starts at locs + n), z[i bs ..]
    for (int i = 0; i < B->nprob && e == cudaSuccess; ++i) {
        double *in = B->d_inputs + B->in_off[i];
        const size_t bytes = (size_t)B->n[i] * sizeof(double);
        const int64_t off = (int64_t)i * bs;
        e = cudaMemcpyAsync(in, locs + off, bytes, cudaMemcpyDefault, B->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(in + B->n[i], locs + n + off, bytes, cudaMemcpyDefault, B->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(in + 2 * B->n[i], z + off, bytes, cudaMemcpyDefault, B->cs);
    }
    e = run_staged(B, us, e);
    if (e != cudaSuccess) {
        egs_batch_destroy(B);
        return cuda_error(e, "egs_loglik_ind");
    }
    if (B->dag && B->h_ctl[1].timeouts > 0) {
        egs_batch_destroy(B);
        return set_error(EGS_ERR_TIMEOUT, "egs_loglik_ind: a dependency wait of the persistent launch ran out of time");
    }
    // fixed-order FP64 sums over the blocks
    double ll = 0.0, ld = 0.0, q = 0.0;
    int64_t fail = -1;
    for (int i = 0; i < B->nprob; ++i) {
        const DevStatus &h = B->h_status[i];
        if (h.fail_index != kNoFail && fail < 0) fail = (int64_t)i * bs + (int64_t)h.fail_index;
        ll += h.result[0];
        ld += h.result[1];
        q += h.result[2];
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->loglik = fail < 0 ? ll : NAN;
        info->logdet = ld;
        info->quad = q;
        info->quad_unrefined = q;
        info->fail_index = fail;
        info->fail_tile = fail >= 0 ? fail / tile : -1;
        info->tile = tile;
        info->band = super_tiles;
        info->launches = B->launches_per_run;
    }
    egs_batch_destroy(B);
    if (fail >= 0) return set_error(EGS_ERR_NOT_PD, "egs_loglik_ind: not positive definite at row %lld", (long long)fail);
    if (out_loglik) *out_loglik = ll;
    return EGS_OK;
}

}  // extern "C"
