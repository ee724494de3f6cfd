// Persistent batched scheduler for FP64 batches: every problem's tile
// algorithm (Algorithm 2: Matern generation, the tile Cholesky of Section 5.2,
// the forward solve with the log-determinant and the dot product, Eq. 1) is
// expanded into one list of tile tasks, and ONE kernel launch executes the
// whole list.  Each CTA repeatedly claims the next task from a global counter
// and, before running it, waits until the tile counters it depends on have
// reached the values the task needs:
//
//   GEN(i, j)       tile (i, j) of Sigma; GEN(i, i) also copies z block i
//   POTRF(k)        needs the k updates of tile (k, k)
//   TRSM(m, k)      needs POTRF(k) and the k updates of tile (m, k)
//   UPDATE(m, n, k) needs TRSM(m, k), TRSM(n, k) and updates 0..k-1 of (m, n)
//                   (so the updates of a tile are applied in step order)
//   TRSV(k)         needs POTRF(k) and the k panel products into z block k
//   GEMV(m, k)      needs TRSV(k), TRSM(m, k) and the earlier products into m
//   FINAL           needs TRSV(T - 1); assembles l (Eq. 1)
//
// Tile counter (i, j) counts 1 for its generation, 1 per update applied and 1
// when it is final (after POTRF or TRSM); vector counter k counts 1 for its
// initial copy, 1 per panel product and 1 when the block solve is done.
//
// The list is built on the host in a topological order (checked on the host
// by replaying it sequentially), so the lowest unfinished task always has its
// dependencies done: a CTA only waits for tasks that running CTAs have
// already claimed, and the schedule cannot deadlock however many CTAs are
// resident.  Problems are aligned at their last step (problem p's step k sits
// at position k + Tmax - T_p), so the largest problems start first and all
// finish together.  Every wait is bounded by %globaltimer; an expired wait
// sets an abort flag that makes every CTA stop claiming tasks, and the run
// reports EGS_ERR_TIMEOUT.  A problem whose Cholesky fails still signals all
// its counters (without doing the work), so the others are not held up.
//
// The tile routines are the ones of the step-synchronous batch and of the
// single-problem FP64 path, applied in the same order to each tile, so every
// l is bitwise equal to the corresponding egs_loglik_ex result.
#include <algorithm>
#include <vector>

#include "batched.cuh"
#include "batched_dag.cuh"
#include "blocks.cuh"
#include "matern.cuh"

namespace egs {

namespace {

enum DagType { D_GEN = 0, D_POTRF, D_TRSM, D_UPDATE, D_TRSV, D_GEMV, D_FINAL };

struct TrsvSmem {
    double yv[256];
    double red[256];
    double D[32][33];
    double ldq[2];
};

// The tasks' shared memory, overlaid: one task runs at a time in a CTA.
struct GenSmem {
    egs_matern_params P;
    double T[EGS_MT_DOUBLES];
};

union DagSmem {
    TrsmSmem<64, double> trsm;
    Trsm32Smem trsm32;
    PotrfSmem<32> potrf32;
    GemmSmem<double> gemm;
    Gemm32Smem gemm32;
    TrsvSmem trsv;
    GenSmem gen;
    double vec[256];
};

struct DagArgs {
    const int4 *tasks;  // x = problem, y = type | (i << 16), z = j | (k << 16), w = unused
    long long ntasks;
    const BatchProblem *probs;
    DagCtl *ctl;
    int b;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 of a CTA: wait until *c >= target.  False if the batch aborted
// (this wait or another one ran out of time).
__device__ bool dag_wait(const unsigned *c, unsigned target, DagCtl *ctl)
{
    if (ld_acquire(c) >= target) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = *(volatile unsigned long long *)&ctl->limit_ns;
    for (;;) {
        __nanosleep(100);
        if (ld_acquire(c) >= target) return true;
        if (*(volatile unsigned *)&ctl->abort) return false;
        if (global_ns() - t0 > limit) {
            atomicAdd(&ctl->timeouts, 1u);
            atomicExch(&ctl->abort, 1u);
            return false;
        }
    }
}

__device__ __forceinline__ unsigned *tile_cnt(const BatchProblem &p, int i, int j)
{
    return p.cnt + tile_linear(i, j);
}

__device__ __forceinline__ unsigned *vec_cnt(const BatchProblem &p, int k)
{
    return p.cnt + (size_t)p.T * (p.T + 1) / 2 + k;
}

// Forward substitution on one diagonal tile, as trsv_fwd_tile but for a CTA
// of 256 threads and b <= 256 (threads >= b own no row; their zeros enter the
// fixed-order trees as exact additions, so the sums are those of a CTA of b
// threads).  Reads go through plain (coherent) loads: the tile and the vector
// were written earlier in the same launch.
__device__ void dag_trsv_fwd(TrsvSmem &sm, const double *L, int b, double *v, double *ld_q)
{
    double(&yv)[256] = sm.yv;
    double(&D)[32][33] = sm.D;
    double *red = sm.red;
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const bool own = i < b;
    const double *Li = L + (size_t)(own ? i : 0) * b;
    double r = own ? v[i] : 0.0;
    for (int cb = 0; cb < b / 32; ++cb) {
        const int c0 = cb * 32;
        for (int e = i; e < 32 * 32; e += 256) D[e >> 5][e & 31] = L[(size_t)(c0 + (e >> 5)) * b + c0 + (e & 31)];
        __syncthreads();
        if (w == cb) {
            for (int jj = 0; jj < 32; ++jj) {
                const double yj = __shfl_sync(0xffffffffu, r, jj) / D[jj][jj];
                if (lane == jj) yv[c0 + jj] = yj;
                if (lane > jj) r = fma(-D[lane][jj], yj, r);
            }
        }
        __syncthreads();
        if (own && i >= c0 + 32) {
            double s = 0.0;
#pragma unroll 8
            for (int jj = 0; jj < 32; ++jj) s = fma(Li[c0 + jj], yv[c0 + jj], s);
            r -= s;
        }
    }
    __syncthreads();
    const double y = own ? yv[i] : 0.0;
    if (own) v[i] = y;
    const double ld = block_sum(own ? log(Li[i]) : 0.0, red);
    __syncthreads();
    const double q = block_sum(y * y, red);
    if (i == 0) {
        ld_q[0] = ld;
        ld_q[1] = q;
    }
    __syncthreads();
}

// out[r] -= L[r][:] . ys for the 64 rows r0..r0+63 (as gemv_rows, plain loads).
__device__ __forceinline__ void dag_gemv_rows(const double *A, int b, int r0, const double *ys, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int rr = 0; rr < 8; ++rr) {
        const int r = r0 + warp * 8 + rr;
        const double *row = A + (size_t)r * b;
        double s = 0.0;
        for (int c = lane; c < b; c += 32) s = fma(row[c], ys[c], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out[r] -= s;
    }
}

__device__ void task_gen(GenSmem &gs, const BatchProblem &pr, int b, int ti, int tj)
{
    egs_matern_params &Ps = gs.P;
    {
        const double *s = reinterpret_cast<const double *>(pr.P);
        double *d = reinterpret_cast<double *>(&Ps);
        for (int i = threadIdx.x; i < (int)(sizeof(egs_matern_params) / sizeof(double)); i += blockDim.x) d[i] = s[i];
        __syncthreads();
    }
    const bool general = Ps.kind == EGS_MATERN_GENERAL;
    if (general) {
        for (int i = threadIdx.x; i < EGS_MT_DOUBLES; i += blockDim.x) gs.T[i] = pr.mtab[i];
        __syncthreads();
    }
    const double *Tab = general ? gs.T : nullptr;
    const int nsub = b >> 6, tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int64_t n = pr.n;
    double *tile = pr.tiles + (size_t)tile_linear(ti, tj) * b * b;
    for (int sub = 0; sub < nsub * nsub; ++sub) {
        const int sr = sub / nsub, sc = sub % nsub;
        const int64_t gj = (int64_t)tj * b + sc * 64 + tx;
        const double xj = gj < n ? pr.X[gj] : 0.0, yj = gj < n ? pr.Y[gj] : 0.0;
        for (int rr = 0; rr < 16; ++rr) {
            const int r = sr * 64 + ty + 4 * rr;
            const int64_t gi = (int64_t)ti * b + r;
            double v;
            if (gi >= n || gj >= n) v = (gi == gj) ? 1.0 : 0.0;
            else if (gi == gj) v = Ps.th1;
            else v = matern_eval(&Ps, loc_dist(&Ps, pr.X[gi], pr.Y[gi], xj, yj) * Ps.inv_th2, Tab);
            tile[(size_t)r * b + sc * 64 + tx] = v;
        }
    }
    if (ti == tj)
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            const int64_t i = (int64_t)ti * b + r;
            pr.zpad[i] = i < n ? pr.z[i] : 0.0;
        }
}

// POTRF of diagonal tile k in one CTA: the 32 x 32 block operations of the
// single-problem diagonal POTRF (chol64.cu) run in its task order -- for each
// block column p, POTRF of block (p, p) (and the zeros right of it), the
// 32-row solves below it, then the updates of the trailing blocks -- so every
// element sees the same operations in the same order and the factor is the
// single evaluation's bit for bit.
__device__ void task_potrf(DagSmem &sm, const BatchProblem &pr, int b, int k)
{
    double *A = pr.tiles + (size_t)tile_linear(k, k) * b * b;
    const int nb = b >> 5;
    for (int p = 0; p < nb; ++p) {
        double *Ap = A + (size_t)p * 32 * b + p * 32;
        if (!potrf_smem_s<32>(sm.potrf32, Ap, b, (int64_t)k * b + p * 32, pr.st)) return;
        for (int e = threadIdx.x; e < 32 * (b - p * 32 - 32); e += 256) {
            const int r = e / (b - p * 32 - 32), c = e % (b - p * 32 - 32);
            Ap[(size_t)r * b + 32 + c] = 0.0;
        }
        __syncthreads();
        for (int m = p + 1; m < nb; ++m) trsm32_s(sm.trsm32, Ap, b, A + (size_t)m * 32 * b + p * 32, b);
        for (int m = p + 1; m < nb; ++m)
            for (int n = p + 1; n <= m; ++n) {
                gemm_sub32_s(sm.gemm32, A + (size_t)m * 32 * b + p * 32, b, A + (size_t)n * 32 * b + p * 32, b, 32,
                             A + (size_t)m * 32 * b + n * 32, b);
                __syncthreads();
            }
    }
}

__device__ void task_trsm(DagSmem &sm, const BatchProblem &pr, int b, int m, int k)
{
    const double *Lkk = pr.tiles + (size_t)tile_linear(k, k) * b * b;
    double *X = pr.tiles + (size_t)tile_linear(m, k) * b * b;
    for (int r0 = 0; r0 < b; r0 += 64) trsm_rows_s<64>(sm.trsm, Lkk, b, X + (size_t)r0 * b, b, b);
}

__device__ void task_update(DagSmem &sm, const BatchProblem &pr, int b, int m, int nc, int k)
{
    const size_t bb = (size_t)b * b;
    const double *Am = pr.tiles + (size_t)tile_linear(m, k) * bb;
    const double *An = pr.tiles + (size_t)tile_linear(nc, k) * bb;
    double *C = pr.tiles + (size_t)tile_linear(m, nc) * bb;
    const int nsub = b >> 6;
    for (int sr = 0; sr < nsub; ++sr)
        for (int sc = 0; sc < nsub; ++sc) {
            if (m == nc && sc > sr) continue;
            gemm_sub64_s(sm.gemm, Am + (size_t)sr * 64 * b, b, An + (size_t)sc * 64 * b, b, b,
                         C + (size_t)sr * 64 * b + sc * 64, b);
        }
}

__device__ void task_trsv(DagSmem &sm, const BatchProblem &pr, int b, int k)
{
    double *ldq = sm.trsv.ldq;
    dag_trsv_fwd(sm.trsv, pr.tiles + (size_t)tile_linear(k, k) * b * b, b, pr.zpad + (size_t)k * b, ldq);
    if (threadIdx.x == 0) {
        pr.partials[k] = ldq[0];
        pr.partials[pr.T + k] = ldq[1];
    }
}

__device__ void task_gemv(DagSmem &sm, const BatchProblem &pr, int b, int m, int k)
{
    double *ys = sm.vec;
    for (int c = threadIdx.x; c < b; c += 256) ys[c] = pr.zpad[(size_t)k * b + c];
    __syncthreads();
    const double *A = pr.tiles + (size_t)tile_linear(m, k) * b * b;
    for (int r0 = 0; r0 < b; r0 += 64) dag_gemv_rows(A, b, r0, ys, pr.zpad + (size_t)m * b);
}

// l from the log-det and dot partials (as k_finalize / kb_finalize).
__device__ void task_final(DagSmem &sm, const BatchProblem &pr)
{
    double *red = sm.vec;
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

// Thread 0: the waits of one task.
__device__ bool task_wait(int type, int i, int j, int k, const BatchProblem &pr, DagCtl *ctl)
{
    switch (type) {
    case D_POTRF: return dag_wait(tile_cnt(pr, k, k), (unsigned)k + 1, ctl);
    case D_TRSM:
        return dag_wait(tile_cnt(pr, k, k), (unsigned)k + 2, ctl) && dag_wait(tile_cnt(pr, i, k), (unsigned)k + 1, ctl);
    case D_UPDATE:
        return dag_wait(tile_cnt(pr, i, k), (unsigned)k + 2, ctl) && dag_wait(tile_cnt(pr, j, k), (unsigned)k + 2, ctl) &&
               dag_wait(tile_cnt(pr, i, j), (unsigned)k + 1, ctl);
    case D_TRSV:
        return dag_wait(tile_cnt(pr, k, k), (unsigned)k + 2, ctl) && dag_wait(vec_cnt(pr, k), (unsigned)k + 1, ctl);
    case D_GEMV:
        return dag_wait(vec_cnt(pr, k), (unsigned)k + 2, ctl) && dag_wait(tile_cnt(pr, i, k), (unsigned)k + 2, ctl) &&
               dag_wait(vec_cnt(pr, i), (unsigned)k + 1, ctl);
    case D_FINAL: return dag_wait(vec_cnt(pr, pr.T - 1), (unsigned)pr.T + 1, ctl);
    default: return true;  // D_GEN
    }
}

// Thread 0, after the task's work: release its counter(s).
__device__ void task_signal(int type, int i, int j, int k, const BatchProblem &pr)
{
    __threadfence();
    switch (type) {
    case D_GEN:
        atomicAdd(tile_cnt(pr, i, j), 1u);
        if (i == j) atomicAdd(vec_cnt(pr, i), 1u);
        break;
    case D_POTRF: atomicAdd(tile_cnt(pr, k, k), 1u); break;
    case D_TRSM: atomicAdd(tile_cnt(pr, i, k), 1u); break;
    case D_UPDATE: atomicAdd(tile_cnt(pr, i, j), 1u); break;
    case D_TRSV: atomicAdd(vec_cnt(pr, k), 1u); break;
    case D_GEMV: atomicAdd(vec_cnt(pr, i), 1u); break;
    default: break;
    }
}

__global__ void __launch_bounds__(256, 2) kb_dag(DagArgs a)
{
    __shared__ int4 s_task;
    __shared__ long long s_idx;
    __shared__ int s_go, s_skip;
    __shared__ DagSmem sm;
    for (;;) {
        if (threadIdx.x == 0) {
            int go = 0;
            if (!*(volatile unsigned *)&a.ctl->abort) {
                const long long t = (long long)atomicAdd(&a.ctl->next, 1ull);
                if (t < a.ntasks) {
                    s_task = a.tasks[t];
                    s_idx = t;
                    go = 1;
                }
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        const int4 tk = s_task;
        const long long idx = s_idx;
        const BatchProblem &pr = a.probs[tk.x];
        const int type = tk.y & 0xFFFF, i = tk.y >> 16, j = tk.z & 0xFFFF, k = tk.z >> 16;
        if (threadIdx.x == 0) {
            s_go = task_wait(type, i, j, k, pr, a.ctl) ? 1 : 0;
            s_skip = failed(pr.st) ? 1 : 0;
        }
        __syncthreads();
        if (!s_go) return;
        if (!s_skip || type == D_FINAL) {
            switch (type) {
            case D_GEN: task_gen(sm.gen, pr, a.b, i, j); break;
            case D_POTRF: task_potrf(sm, pr, a.b, k); break;
            case D_TRSM: task_trsm(sm, pr, a.b, i, k); break;
            case D_UPDATE: task_update(sm, pr, a.b, i, j, k); break;
            case D_TRSV: task_trsv(sm, pr, a.b, k); break;
            case D_GEMV: task_gemv(sm, pr, a.b, i, k); break;
            case D_FINAL: task_final(sm, pr); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && idx != *(volatile long long *)&a.ctl->withhold) task_signal(type, i, j, k, pr);
    }
}

inline int4 pack(int prob, int type, int i, int j, int k) { return make_int4(prob, type | (i << 16), j | (k << 16), 0); }

}  // namespace

egs_status dag_plan(const std::vector<int> &T, int b, std::vector<int4> &tasks, std::vector<size_t> &cnt_off,
                    size_t &ncounters)
{
    const int np = (int)T.size();
    if (b > 256 || b % 64) return set_error(EGS_ERR_ARG, "persistent batch: tile %d must be 64, 128, 192 or 256", b);
    int Tmax = 0;
    cnt_off.resize(np);
    ncounters = 0;
    for (int p = 0; p < np; ++p) {
        if (T[p] > 32767) return set_error(EGS_ERR_ARG, "persistent batch: %d tiles per side is too many", T[p]);
        Tmax = std::max(Tmax, T[p]);
        cnt_off[p] = ncounters;
        ncounters += (size_t)T[p] * (T[p] + 1) / 2 + T[p];
    }
    tasks.clear();
    // position key = k + Tmax - T_p; generation at key - 1.  Within a key:
    // POTRF, TRSM, UPDATE, TRSV, GEMV, FINAL, each over all problems.
    for (int key = -1; key < Tmax; ++key) {
        for (int p = 0; p < np; ++p) {
            const int k = key - (Tmax - T[p]) + 1;  // generation precedes step 0
            if (k == 0)
                for (int i = 0; i < T[p]; ++i)
                    for (int j = 0; j <= i; ++j) tasks.push_back(pack(p, D_GEN, i, j, 0));
        }
        for (int rank = 0; rank < 6; ++rank)
            for (int p = 0; p < np; ++p) {
                const int k = key - (Tmax - T[p]);
                if (k < 0 || k >= T[p]) continue;
                const int Tp = T[p];
                switch (rank) {
                case 0: tasks.push_back(pack(p, D_POTRF, k, k, k)); break;
                case 1:
                    for (int m = k + 1; m < Tp; ++m) tasks.push_back(pack(p, D_TRSM, m, k, k));
                    break;
                case 2:
                    for (int m = k + 1; m < Tp; ++m)
                        for (int n = k + 1; n <= m; ++n) tasks.push_back(pack(p, D_UPDATE, m, n, k));
                    break;
                case 3: tasks.push_back(pack(p, D_TRSV, k, k, k)); break;
                case 4:
                    for (int m = k + 1; m < Tp; ++m) tasks.push_back(pack(p, D_GEMV, m, k, k));
                    break;
                case 5:
                    if (k == Tp - 1) tasks.push_back(pack(p, D_FINAL, 0, 0, 0));
                    break;
                }
            }
    }
    // Replay the list sequentially: every wait must already hold from the
    // tasks before it (so the ordered claiming cannot deadlock), and every
    // counter must end at its final value.
    std::vector<unsigned> c(ncounters, 0);
    auto tc = [&](int p, int i, int j) -> unsigned & { return c[cnt_off[p] + (size_t)i * (i + 1) / 2 + j]; };
    auto vc = [&](int p, int k) -> unsigned & { return c[cnt_off[p] + (size_t)T[p] * (T[p] + 1) / 2 + k]; };
    for (size_t t = 0; t < tasks.size(); ++t) {
        const int4 tk = tasks[t];
        const int p = tk.x, type = tk.y & 0xFFFF, i = tk.y >> 16, j = tk.z & 0xFFFF, k = tk.z >> 16;
        const unsigned uk = (unsigned)k;
        bool ok = true;
        switch (type) {
        case D_GEN: ++tc(p, i, j); if (i == j) ++vc(p, i); break;
        case D_POTRF: ok = tc(p, k, k) >= uk + 1; ++tc(p, k, k); break;
        case D_TRSM: ok = tc(p, k, k) >= uk + 2 && tc(p, i, k) >= uk + 1; ++tc(p, i, k); break;
        case D_UPDATE:
            ok = tc(p, i, k) >= uk + 2 && tc(p, j, k) >= uk + 2 && tc(p, i, j) >= uk + 1;
            ++tc(p, i, j);
            break;
        case D_TRSV: ok = tc(p, k, k) >= uk + 2 && vc(p, k) >= uk + 1; ++vc(p, k); break;
        case D_GEMV: ok = vc(p, k) >= uk + 2 && tc(p, i, k) >= uk + 2 && vc(p, i) >= uk + 1; ++vc(p, i); break;
        case D_FINAL: ok = vc(p, T[p] - 1) >= (unsigned)T[p] + 1; break;
        }
        if (!ok) return set_error(EGS_ERR_ARG, "persistent batch: task %zu of the plan is not in dependency order", t);
    }
    for (int p = 0; p < np; ++p)
        for (int i = 0; i < T[p]; ++i) {
            if (vc(p, i) != (unsigned)i + 2) return set_error(EGS_ERR_ARG, "persistent batch: incomplete solve plan");
            for (int j = 0; j <= i; ++j)
                if (tc(p, i, j) != (unsigned)j + 2) return set_error(EGS_ERR_ARG, "persistent batch: incomplete plan");
        }
    return EGS_OK;
}

int dag_grid()
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kb_dag, 256, 0) != cudaSuccess || per < 1) per = 1;
    return sms * per;
}

cudaError_t dag_enqueue(const int4 *d_tasks, long long ntasks, const BatchProblem *d_probs, DagCtl *d_ctl, int b,
                        int grid, cudaStream_t s)
{
    DagArgs a{d_tasks, ntasks, d_probs, d_ctl, b};
    kb_dag<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace egs
