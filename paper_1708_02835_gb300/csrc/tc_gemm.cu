// Tensor-core (tcgen05) trailing update of the mixed-precision tile Cholesky,
// the dominant contraction of Algorithm 2's dpotrf (Section 5.2, GEMM/SYRK
// tasks):  C_mn -= P_m P_n^T  for every tile T > m >= n > k at step k, where
// P_m is the factored panel tile (m, k) stored in the MMA operand format
// (TF32-rounded FP32, split-TF32 hi/lo copies, or BF16) by the TRSM stage.
//
// A persistent kernel (one CTA per SM) loops over 128 x 256 blocks of the
// output tiles: one elected thread of warp 0 streams 128-byte-wide K slices of
// the two operands into a 4-stage shared-memory ring with TMA (128-byte
// swizzle); one thread of warp 1 issues tcgen05.mma (M = 128, N = 256) into
// one of two 256-column FP32 accumulators in TMEM and releases each stage with
// tcgen05.commit; eight epilogue warps drain the other accumulator with
// tcgen05.ld and subtract it from the output tile -- by a TMA reduce-add for
// FP32 tiles, by a read-modify-write in FP64 for band tiles.  No cluster
// multicast is used.
#include "egs_internal.cuh"
#include "tc_common.cuh"

#include <cudaTypedefs.h>

namespace egs {

namespace {

// 4 stages of 48 KB keep about 1.3 us of operands in flight (at the tensor
// peak one stage is consumed in ~0.33 us); each epilogue warp then has one
// 4 KB staging box for its TMA reduces.
constexpr int BM = 128, BN = 256, STAGES = 4;
// SMs the bulk update leaves to the lookahead chain (POTRF / TRSM / band
// update of the next step on the side stream).  While the bulk update is
// several times longer than that chain (many work items), 8 SMs keep the
// chain off the critical path and the tensor cores get the rest.
constexpr int kReserveSms = 24;
constexpr int kReserveSmsLong = 8;
constexpr int64_t kLongBulkItems = 72000;
constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
constexpr int EPI_WARPS = 8;
constexpr int STAGE_C = 32 * 32 * 4;  // one 32 x 32 FP32 box staged for the TMA reduce
// Operand formats: 1 = BF16, 2 = TF32 (one box of A and one of B per stage,
// 4 stages of 48 KB), 3 = split TF32 (A and B rows [hi | lo] over K = 2b: a
// stage holds the hi and lo boxes of A and of B for one 32-element K slice,
// 2 stages of 96 KB, and feeds lo hi' + hi lo' + hi hi' into the accumulator),
// 4 = split FP16 (the same with FP16 halves of rows scaled by a power of two
// per row, 64-element K slices, FP16 MMAs at twice the TF32 rate; the
// epilogue multiplies by the row scales of both operands, exactly).
template <int FMT>
struct Cfg {
    static constexpr int STAGES_ = FMT >= 3 ? 2 : STAGES;
    static constexpr int STAGE_BYTES = FMT >= 3 ? 2 * (A_BYTES + B_BYTES) : A_BYTES + B_BYTES;
    static constexpr int SMEM_BYTES = STAGES_ * STAGE_BYTES + EPI_WARPS * STAGE_C + 1024;
    static_assert(SMEM_BYTES + 512 <= 232448, "dynamic + static shared memory must fit 227 KB");
};
constexpr uint32_t TMEM_COLS = 256;

struct WorkItem {
    int m, n;    // output tile (update) / unused (dense)
    int rb, cb;  // 128-row block, 256-column block
    int ya, yb;  // TMA row coordinates of the A and B boxes
};

// Trailing update of step k over the lower-tile storage: the output tiles
// (m, n) with m >= n >= col0 (one_col: only n = col0).  Panel tile m of
// step k is operand row block m - k - 1.  skip_band: leave every band output
// (m - n < band) to the FP64 kernels (split-TF32 mode).
//
// Tiles are visited by blocks of kColBlock columns: for each block, its
// triangle (rows inside the block) then every lower row, kColBlock tiles per
// row.  The persistent CTAs, which work on consecutive items together, then
// share one block's B operand tiles (48 MB in split TF32 at b = 512, resident
// in the 129 MB L2) while the A rows stream past, instead of needing every B
// tile of a row at once.  Measured at n = 102,400: 8 columns 677 TFLOP/s,
// 16 columns 696, 32 columns 666 (row order: 648).
constexpr int kColBlock = 16;
struct UpdateWork {
    Tiles tl;
    int k;
    int col0;
    int one_col;
    int skip_band;
    const float *rs;  // split FP16: the power-of-two scale of every panel row
    int xband;        // skip_band: outputs with m - n < xband are done by the FP64-accurate kernels
    __device__ float row_scale(int y) const { return rs[y]; }
    __device__ bool decode(int64_t bid, WorkItem &w) const
    {
        const int nrb = tl.b / BM, ncb = tl.b / BN, per = nrb * ncb;
        int64_t t = bid / per;
        const int blk = (int)(bid % per);
        if (one_col) {
            w.m = col0 + (int)t;
            w.n = col0;
        } else {
            // column block c_lo .. c_lo + wd - 1: wd (wd + 1) / 2 triangle tiles,
            // then (T - c_lo - wd) rows of wd tiles
            int c_lo = col0;
            while (true) {
                const int wd = min(kColBlock, tl.T - c_lo);
                if (wd <= 0) return false;  // past the last tile (not reached for valid items)
                const int64_t tri = (int64_t)wd * (wd + 1) / 2;
                const int64_t cnt = tri + (int64_t)(tl.T - c_lo - wd) * wd;
                if (t < cnt) {
                    if (t < tri) {
                        int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
                        while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
                        while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
                        w.m = c_lo + ii;
                        w.n = c_lo + (int)(t - (int64_t)ii * (ii + 1) / 2);
                    } else {
                        const int64_t u = t - tri;
                        w.m = c_lo + wd + (int)(u / wd);
                        w.n = c_lo + (int)(u % wd);
                    }
                    break;
                }
                t -= cnt;
                c_lo += wd;
            }
        }
        w.rb = blk / ncb;
        w.cb = blk % ncb;
        if (w.m - k < tl.band && w.n - k < tl.band) return false;         // FP64 band x band: done in FP64
        if (skip_band && w.m - w.n < xband) return false;                // FP64-accurate output: done elsewhere
        if (w.m == w.n && w.cb * BN > w.rb * BM + BM - 1) return false;  // strictly above the diagonal
        w.ya = (w.m - k - 1) * tl.b + w.rb * BM;
        w.yb = (w.n - k - 1) * tl.b + w.cb * BN;
        return true;
    }
    // 64 consecutive columns from two accumulator slices; all loads of the
    // old values are issued before any store so they overlap in flight.
    __device__ void store2(const WorkItem &w, int r, int c0, const float (&v0)[32], const float (&v1)[32]) const
    {
        const size_t row = (size_t)(w.rb * BM + r), col = (size_t)(w.cb * BN + c0);
        if (tl.is64(w.m, w.n)) {
            double *C = tl.t64(w.m, w.n) + row * tl.b + col;
            double2 c[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) c[i] = *reinterpret_cast<const double2 *>(C + 2 * i);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                c[i].x -= (double)v0[2 * i];
                c[i].y -= (double)v0[2 * i + 1];
                c[16 + i].x -= (double)v1[2 * i];
                c[16 + i].y -= (double)v1[2 * i + 1];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) *reinterpret_cast<double2 *>(C + 2 * i) = c[i];
        } else {
            float *C = tl.t32(w.m, w.n) + row * tl.b + col;
            float4 c[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) c[i] = *reinterpret_cast<const float4 *>(C + 4 * i);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                c[i].x -= v0[4 * i];
                c[i].y -= v0[4 * i + 1];
                c[i].z -= v0[4 * i + 2];
                c[i].w -= v0[4 * i + 3];
                c[8 + i].x -= v1[4 * i];
                c[8 + i].y -= v1[4 * i + 1];
                c[8 + i].z -= v1[4 * i + 2];
                c[8 + i].w -= v1[4 * i + 3];
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) *reinterpret_cast<float4 *>(C + 4 * i) = c[i];
        }
    }
    // FP32 output tiles take the TMA reduce path: row of the 2-D view of the
    // off-band tile array where output row r of this item lives.
    static constexpr bool kReduce = true;
    __device__ bool reduce_here(const WorkItem &w) const { return !tl.is64(w.m, w.n); }
    __device__ int reduce_row(const WorkItem &w, int r) const
    {
        const int64_t q = w.m - tl.band;
        const int64_t idx = q * (q + 1) / 2 + w.n;
        return (int)(idx * tl.b + w.rb * BM + r);
    }
    __device__ int reduce_col(const WorkItem &w, int c0) const { return w.cb * BN + c0; }
    __device__ void store(const WorkItem &w, int r, int c0, const float (&v)[32]) const
    {
        const size_t row = (size_t)(w.rb * BM + r), col = (size_t)(w.cb * BN + c0);
        if (tl.is64(w.m, w.n)) {
            double *C = tl.t64(w.m, w.n) + row * tl.b + col;
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                double2 c = *reinterpret_cast<double2 *>(C + i);
                c.x -= (double)v[i];
                c.y -= (double)v[i + 1];
                *reinterpret_cast<double2 *>(C + i) = c;
            }
        } else {
            float *C = tl.t32(w.m, w.n) + row * tl.b + col;
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                float4 c = *reinterpret_cast<float4 *>(C + i);
                c.x -= v[i];
                c.y -= v[i + 1];
                c.z -= v[i + 2];
                c.w -= v[i + 3];
                *reinterpret_cast<float4 *>(C + i) = c;
            }
        }
    }
};

// FP32 mode, off-band panel TRSM of step k as a product with the inverse
// diagonal tile: X_mk = A_mk L_kk^-T = A_mk W^T, W = L_kk^-1, for the tiles
// m = m0 .. T - 1.  A rows: the unsolved tiles in split-TF32 layout [hi | lo]
// at operand row (m - k - 1) b (the spare panel buffer of the step); B rows:
// W in the same layout (b rows of 2b floats).  The accumulator is X itself,
// stored over A_mk (each output block is written by exactly one item, and
// the operands live in other buffers, so there is no read-after-write race).
struct TrsmWork {
    Tiles tl;
    int k, m0;
    static constexpr bool kReduce = false;
    __device__ bool reduce_here(const WorkItem &) const { return false; }
    __device__ int reduce_row(const WorkItem &, int) const { return 0; }
    __device__ int reduce_col(const WorkItem &, int) const { return 0; }
    __device__ bool decode(int64_t bid, WorkItem &w) const
    {
        const int ncb = tl.b / BN, per = (tl.b / BM) * ncb;
        const int blk = (int)(bid % per);
        w.m = m0 + (int)(bid / per);
        w.n = k;
        w.rb = blk / ncb;
        w.cb = blk % ncb;
        w.ya = (w.m - k - 1) * tl.b + w.rb * BM;
        w.yb = w.cb * BN;
        return true;
    }
    __device__ void store2(const WorkItem &w, int r, int c0, const float (&v0)[32], const float (&v1)[32]) const
    {
        float *X = tl.t32(w.m, k) + (size_t)(w.rb * BM + r) * tl.b + w.cb * BN + c0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            *reinterpret_cast<float4 *>(X + 4 * i) = make_float4(v0[4 * i], v0[4 * i + 1], v0[4 * i + 2], v0[4 * i + 3]);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            *reinterpret_cast<float4 *>(X + 32 + 4 * i) =
                make_float4(v1[4 * i], v1[4 * i + 1], v1[4 * i + 2], v1[4 * i + 3]);
    }
};

// Plain C = A B^T (A: M x K, B: N x K, row-major), used to test the pipeline.
struct DenseWork {
    float *C;
    int N;  // columns of C
    int nrb, ncb;
    static constexpr bool kReduce = false;
    __device__ bool reduce_here(const WorkItem &) const { return false; }
    __device__ int reduce_row(const WorkItem &, int) const { return 0; }
    __device__ int reduce_col(const WorkItem &, int) const { return 0; }
    __device__ bool decode(int64_t bid, WorkItem &w) const
    {
        w.rb = (int)(bid / ncb);
        w.cb = (int)(bid % ncb);
        w.m = w.n = 0;
        w.ya = w.rb * BM;
        w.yb = w.cb * BN;
        return true;
    }
    __device__ void store2(const WorkItem &w, int r, int c0, const float (&v0)[32], const float (&v1)[32]) const
    {
        store(w, r, c0, v0);
        store(w, r, c0 + 32, v1);
    }
    __device__ void store(const WorkItem &w, int r, int c0, const float (&v)[32]) const
    {
        float *Cp = C + (size_t)(w.rb * BM + r) * N + w.cb * BN + c0;
#pragma unroll
        for (int i = 0; i < 32; i += 4) *reinterpret_cast<float4 *>(Cp + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
};

// Persistent kernel: one CTA per SM.  Warp 0 (one lane) claims work items
// from a global counter (atomicAdd; zeroed before each launch at err + 2),
// posts each item to the other warps through a 4-slot ring in shared memory
// (-1 ends), and streams its operands through the 4-stage ring; warp 1 (one lane) issues
// the MMAs of item t into TMEM accumulator t % 2 (two 256-column buffers);
// warps 2-9 drain accumulator t % 2 while the MMAs of item t + 1 run.
// FMT: 2 = TF32 (K-slice 8 per MMA), 1 = BF16 (K-slice 16 per MMA).
constexpr int NUM_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int RING = 4;           // work items fetched ahead by the producer
constexpr uint32_t TMEM_COLS2 = 2 * TMEM_COLS;

template <int FMT, class Work>
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          const __grid_constant__ CUtensorMap mapC, Work work, int64_t nitems, int kchunks, int *err,
          int64_t withhold)
{
    constexpr int STAGES = Cfg<FMT>::STAGES_;
    constexpr int STAGE_BYTES = Cfg<FMT>::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
    __shared__ uint64_t rfull[RING], rempty[RING];
    __shared__ int64_t ring[RING];  // work items in the order the producer fetched them; -1 ends
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int last_chunk[STAGES];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
            last_chunk[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 8);
        }
        for (int r = 0; r < RING; ++r) {
            tc::mbar_init(&rfull[r], 1);
            tc::mbar_init(&rempty[r], 1 + 8);  // the MMA lane and the eight epilogue warps
        }
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    unsigned long long *next = reinterpret_cast<unsigned long long *>(err + 2);
    if (warp == 0) tc::tmem_alloc(&tmem_base, TMEM_COLS2);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = tmem_base;
    constexpr int KELEMS = (FMT == 1 || FMT == 4) ? 64 : 32;  // elements per 128-byte row slice
    const int klo = kchunks * KELEMS;                         // FMT 3 / 4: K offset of the lo half of a row

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_tmap(&mapA);
            tc::prefetch_tmap(&mapB);
            int g = 0, r = 0;
            // dynamic schedule: the next unclaimed item (CTAs that start late,
            // behind kernels of the other stream, simply take fewer).  The
            // claim of item t + 1 is issued before item t's operand loads, so
            // the atomic's round trip overlaps them instead of opening a gap
            // in the ring at every item boundary.
            int64_t claimed = (int64_t)atomicAdd(next, 1ull);
            while (!abort_flag) {
                const int64_t item = claimed;
                WorkItem wi;
                const bool valid = item < nitems && work.decode(item, wi);
                if (item < nitems && !valid) {
                    claimed = (int64_t)atomicAdd(next, 1ull);
                    continue;
                }
                const int slot = r % RING;
                if (!tc::mbar_wait(&rempty[slot], ((uint32_t)(r / RING) & 1u) ^ 1u, &abort_flag)) break;
                ring[slot] = valid ? item : -1;
                tc::mbar_arrive(&rfull[slot]);
                ++r;
                if (!valid) break;
                claimed = (int64_t)atomicAdd(next, 1ull);
                for (int c = 0; c < kchunks; ++c, ++g) {
                    const int s = g % STAGES;
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    // test hook: the stage `withhold` is never loaded, so the
                    // MMA warp's bounded wait for it runs out and the kernel
                    // unwinds (-1 in every real launch)
                    if (g == withhold) continue;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, &abort_flag)) break;
                    tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    uint8_t *st = smem + s * STAGE_BYTES;
                    if (FMT >= 3) {
                        tc::tma_load_2d(&mapA, &full[s], st, c * KELEMS, wi.ya);                    // A hi
                        tc::tma_load_2d(&mapA, &full[s], st + A_BYTES, klo + c * KELEMS, wi.ya);    // A lo
                        tc::tma_load_2d(&mapB, &full[s], st + 2 * A_BYTES, c * KELEMS, wi.yb);      // B hi
                        tc::tma_load_2d(&mapB, &full[s], st + 2 * A_BYTES + B_BYTES, klo + c * KELEMS, wi.yb);  // B lo
                    } else {
                        tc::tma_load_2d(&mapA, &full[s], st, c * KELEMS, wi.ya);
                        tc::tma_load_2d(&mapB, &full[s], st + A_BYTES, c * KELEMS, wi.yb);
                    }
                    last_chunk[s] = g;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // instruction formats: 0 = FP16, 1 = BF16 (kind::f16), 2 = TF32 (kind::tf32)
            constexpr uint32_t idesc = tc::idesc_f32acc(BM, BN, FMT == 3 ? 2 : (FMT == 4 ? 0 : FMT));
            int g = 0, t = 0, r = 0;
            while (!abort_flag) {
                const int slot = r % RING;
                if (!tc::mbar_wait(&rfull[slot], (uint32_t)(r / RING) & 1u, &abort_flag)) break;
                const int64_t item = ring[slot];
                tc::mbar_arrive(&rempty[slot]);
                ++r;
                if (item < 0) break;
                const int buf = t & 1;
                const uint32_t use = (uint32_t)(t >> 1);
                if (!tc::mbar_wait(&tempty[buf], (use & 1u) ^ 1u, &abort_flag)) break;
                tc::tc_fence_after();
                const uint32_t d = tbase + (uint32_t)buf * TMEM_COLS;
                for (int c = 0; c < kchunks; ++c, ++g) {
                    const int s = g % STAGES;
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (!tc::mbar_wait(&full[s], ph, &abort_flag)) break;
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(smem + s * STAGE_BYTES);
                    if (FMT >= 3) {
                        // lo hi' + hi lo' + hi hi' of every K step (8 TF32 or 16
                        // FP16 elements, 32 bytes): the two small cross terms
                        // enter before the large product
                        const uint32_t alo = a0 + A_BYTES, bhi = a0 + 2 * A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (FMT == 3) {
                                tc::mma_tf32(d, tc::desc_sw128(alo + 32 * j), tc::desc_sw128(bhi + 32 * j), idesc,
                                             (c | j) != 0);
                                tc::mma_tf32(d, tc::desc_sw128(a0 + 32 * j), tc::desc_sw128(blo + 32 * j), idesc, 1u);
                                tc::mma_tf32(d, tc::desc_sw128(a0 + 32 * j), tc::desc_sw128(bhi + 32 * j), idesc, 1u);
                            } else {
                                tc::mma_f16(d, tc::desc_sw128(alo + 32 * j), tc::desc_sw128(bhi + 32 * j), idesc,
                                            (c | j) != 0);
                                tc::mma_f16(d, tc::desc_sw128(a0 + 32 * j), tc::desc_sw128(blo + 32 * j), idesc, 1u);
                                tc::mma_f16(d, tc::desc_sw128(a0 + 32 * j), tc::desc_sw128(bhi + 32 * j), idesc, 1u);
                            }
                        }
                    } else {
                        const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint64_t ad = tc::desc_sw128(a0 + 32 * j);
                            const uint64_t bd = tc::desc_sw128(b0 + 32 * j);
                            if (FMT == 2) tc::mma_tf32(d, ad, bd, idesc, (c | j) != 0);
                            else tc::mma_f16(d, ad, bd, idesc, (c | j) != 0);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&tfull[buf]);
                ++t;
            }
        }
    } else {
        // epilogue warps 2..9: warp w reads TMEM lanes 32 (w % 4) .. + 31 and
        // one half of the 256 columns (warps 2..5 the first, 6..9 the second).
        // FP32 outputs: -acc is staged in shared memory (128-byte swizzle) and
        // added to C by a TMA reduce, so the SM never waits on reading C;
        // FP64 outputs are read-modify-written from registers.
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint8_t *stage = smem + STAGES * STAGE_BYTES + (warp - 2) * STAGE_C;  // after the operand ring
        int t = 0, issued = 0, r = 0;
        while (true) {
            const int slot = r % RING;
            const bool got = tc::mbar_wait(&rfull[slot], (uint32_t)(r / RING) & 1u, &abort_flag);
            if (!__all_sync(0xffffffffu, got && !abort_flag)) break;
            const int64_t item = ring[slot];
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&rempty[slot]);
            ++r;
            if (item < 0) break;
            WorkItem wi;
            work.decode(item, wi);
            const int buf = t & 1;
            const uint32_t use = (uint32_t)(t >> 1);
            const bool ok = tc::mbar_wait(&tfull[buf], use & 1u, &abort_flag);
            tc::tc_fence_after();
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) break;
            const uint32_t d = tbase + (uint32_t)buf * TMEM_COLS + lane_base;
            if (Work::kReduce && work.reduce_here(wi)) {
                const int y = work.reduce_row(wi, q * 32);
                float sr = 1.0f;
                if constexpr (FMT == 4) sr = work.row_scale(wi.ya + q * 32 + lane);
#pragma unroll 1
                for (int cc = half * (BN / 64); cc < (half + 1) * (BN / 64); ++cc) {
                    float v[32];
                    tc::tmem_ld32(d + (uint32_t)(cc * 32), v);
                    if constexpr (FMT == 4) {
                        // the products of scaled rows times both powers of two (exact)
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] *= sr * work.row_scale(wi.yb + cc * 32 + j);
                    }
                    uint8_t *sb = stage;
                    if (issued >= 1 && lane == 0) tc::bulk_wait_read<0>();  // the previous box has been read
                    __syncwarp();
                    // row `lane`, 16-byte chunk j at chunk position j ^ (lane & 7)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4 *>(sb + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                            make_float4(-v[4 * j], -v[4 * j + 1], -v[4 * j + 2], -v[4 * j + 3]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tc::tma_reduce_add_2d(&mapC, sb, work.reduce_col(wi, cc * 32), y);
                        tc::bulk_commit();
                    }
                    ++issued;
                }
            } else {
#pragma unroll 1
                for (int cc = half * (BN / 64); cc < (half + 1) * (BN / 64); cc += 2) {
                    float v0[32], v1[32];
                    tc::tmem_ld32(d + (uint32_t)(cc * 32), v0);
                    tc::tmem_ld32(d + (uint32_t)(cc * 32 + 32), v1);
                    work.store2(wi, q * 32 + lane, cc * 32, v0, v1);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
            ++t;
        }
        if (lane == 0) tc::bulk_wait_all();  // every reduce issued by this warp has landed
        __syncwarp();
    }
    __syncwarp();  // lane 0 of the producer / MMA warps rejoins its warp here
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        // let every TMA load that was issued land before the CTA exits
        for (int s = 0; s < STAGES; ++s)
            if (last_chunk[s] >= 0) {
                volatile int dummy = 0;
                tc::mbar_wait(&full[s], (uint32_t)(last_chunk[s] / STAGES) & 1u, &dummy);
            }
        atomicExch(err, 1);
    }
    tc::tc_fence_after();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS2);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D map over a row-major [rows][inner] array, box {128 bytes of K, box_rows}.
cudaError_t make_map(CUtensorMap *m, const void *base, int fmt, uint64_t inner, uint64_t rows, uint32_t box_rows)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const uint32_t esz = (fmt == 1 || fmt == 4) ? 2 : 4;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * esz};
    cuuint32_t box[2] = {128u / esz, box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                  : (fmt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
    CUresult r = fn(m, dt, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    }
    return sms;
}

// reserve > 0 leaves that many SMs free for kernels on other streams (the
// factorisation's critical chain runs beside the update).
template <int FMT, class Work>
cudaError_t launch_gemm(const CUtensorMap &ma, const CUtensorMap &mb, const CUtensorMap &mc, const Work &w,
                        int64_t items, int kchunks, int *err, cudaStream_t s, int reserve = 0, int64_t withhold = -1)
{
    constexpr int SMEM_BYTES = Cfg<FMT>::SMEM_BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<FMT, Work>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int64_t ctas = num_sms() - reserve > 1 ? num_sms() - reserve : 1;
    const int64_t grid = items < ctas ? items : ctas;
    // err[0] is the error flag; the 8 bytes at err + 2 hold the work counter
    e = cudaMemsetAsync(err + 2, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_tc_gemm<FMT, Work><<<(unsigned)grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, mc, w, items, kchunks, err,
                                                                         withhold);
    return cudaGetLastError();
}

}  // namespace

// Map over the off-band FP32 tile array viewed as rows x b floats, box
// 32 x 32 with the 128-byte swizzle: the target of the epilogue's TMA reduce.
cudaError_t make_offband_map(const float *f32, int b, size_t ntiles, CUtensorMap *mapC)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const uint64_t rows = (uint64_t)(ntiles > 0 ? ntiles : 1) * (uint64_t)b;
    cuuint64_t dims[2] = {(cuuint64_t)b, rows};
    cuuint64_t strides[1] = {(cuuint64_t)b * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(mapC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(f32), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t panel_buffer_bytes(int b, int T, int fmt)
{
    const size_t elems = (size_t)(T > 1 ? T - 1 : 1) * (size_t)b * (size_t)b;
    if (fmt == 3) return 2 * elems * sizeof(float);
    return elems * (fmt == 1 ? 2 : 4);
}

// Panel maps for the trailing update: the panel buffer holds rows
// (T - 1) * b of K = b operand elements (fmt 3 / 4: K = 2b, [hi | lo]); the
// A and B maps view the same rows with boxes of 128 and 256 rows.
cudaError_t make_panel_maps(const void *panel, int fmt, int b, int T, CUtensorMap *mapA, CUtensorMap *mapB)
{
    const uint64_t rows = (uint64_t)(T > 1 ? T - 1 : 1) * (uint64_t)b;
    const uint64_t K = fmt >= 3 ? 2 * (uint64_t)b : (uint64_t)b;
    cudaError_t e = make_map(mapA, panel, fmt, K, rows, BM);
    if (e == cudaSuccess) e = make_map(mapB, panel, fmt, K, rows, BN);
    return e;
}

// Map over W = L_kk^-1 in split-TF32 layout (b rows of [hi | lo], 2b floats).
cudaError_t make_trsm_w_map(const float *wsp, int b, CUtensorMap *mapW)
{
    return make_map(mapW, wsp, 3, 2 * (uint64_t)b, (uint64_t)b, BN);
}

cudaError_t launch_trsm_tc(const CUtensorMap &mapA, const CUtensorMap &mapW, const CUtensorMap &mapC, const Tiles &tl,
                           int k, int m0, int *err, cudaStream_t s, KernelTimer *kt)
{
    const int64_t nf = tl.T - m0;
    if (nf <= 0) return cudaSuccess;
    const int64_t items = nf * (tl.b / BM) * (tl.b / BN);
    TrsmWork w{tl, k, m0};
    if (kt) kt->begin(KC_TRSM, s);
    // a few SMs stay free for the FP64 band update of the step on the side stream
    cudaError_t e = launch_gemm<3>(mapA, mapW, mapC, w, items, tl.b / 32, err, s, kReserveSmsLong);
    if (kt) kt->end(KC_TRSM, s);
    return e;
}

cudaError_t launch_update_tc(const CUtensorMap &mapA, const CUtensorMap &mapB, const CUtensorMap &mapC, int fmt,
                             const Tiles &tl, int k, int *err, cudaStream_t s, KernelTimer *kt, int part,
                             const float *rs, int xband)
{
    // part 0: every trailing tile; 1: column k + 1 only; 2: columns k + 2 .. T - 1
    const int64_t r = tl.T - k - 1;
    int64_t ntiles = 0;
    UpdateWork w{tl, k, k + 1, 0, fmt >= 3 ? 1 : 0, rs, xband > tl.band ? xband : tl.band};
    if (part == 0) ntiles = r * (r + 1) / 2;
    else if (part == 1) {
        ntiles = r;
        w.one_col = 1;
    } else {
        ntiles = (r - 1) * r / 2;
        w.col0 = k + 2;
    }
    if (ntiles <= 0) return cudaSuccess;
    const int64_t blocks = ntiles * (tl.b / BM) * (tl.b / BN);
    // split TF32 / FP16 (fmt 3 / 4): three products per K slice of the [hi | lo] rows
    const int kchunks = tl.b / ((fmt == 1 || fmt == 4) ? 64 : 32);
    cudaError_t e;
    if (kt) kt->begin(KC_UPDATE, s);
    const int reserve = (part != 2) ? 0 : (blocks >= kLongBulkItems ? kReserveSmsLong : kReserveSms);
    if (fmt == 4) e = launch_gemm<4>(mapA, mapB, mapC, w, blocks, kchunks, err, s, reserve);
    else if (fmt == 3) e = launch_gemm<3>(mapA, mapB, mapC, w, blocks, kchunks, err, s, reserve);
    else if (fmt == 2) e = launch_gemm<2>(mapA, mapB, mapC, w, blocks, kchunks, err, s, reserve);
    else e = launch_gemm<1>(mapA, mapB, mapC, w, blocks, kchunks, err, s, reserve);
    if (kt) kt->end(KC_UPDATE, s);
    return e;
}

}  // namespace egs

using namespace egs;

static egs_status tc_gemm_test(const void *A, const void *B, int32_t M, int32_t N, int32_t K, egs_precision p,
                               float *C, int64_t withhold, void *stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || M % BM || N % BN || K % 64)
        return set_error(EGS_ERR_ARG, "egs_tc_gemm_test: M %% 128, N %% 256, K %% 64 must be 0");
    if (p != EGS_MIX_TF32 && p != EGS_MIX_BF16)
        return set_error(EGS_ERR_ARG, "egs_tc_gemm_test: precision must be EGS_MIX_TF32 or EGS_MIX_BF16");
    const int fmt = (p == EGS_MIX_TF32) ? 2 : 1;
    cudaStream_t s = (cudaStream_t)stream;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, A, fmt, (uint64_t)K, (uint64_t)M, BM);
    if (e == cudaSuccess) e = make_map(&mb, B, fmt, (uint64_t)K, (uint64_t)N, BN);
    if (e != cudaSuccess) return set_error(EGS_ERR_CUDA, "egs_tc_gemm_test: tensor map encoding failed");
    int *err = nullptr;
    const Allocator Al = current_allocator();
    e = dev_alloc(Al, (void **)&err, 256, s);  // error flag + work counter
    if (e != cudaSuccess) return set_error(EGS_ERR_OOM, "egs_tc_gemm_test: workspace");
    cudaMemsetAsync(err, 0, 16, s);
    DenseWork w{C, N, M / BM, N / BN};
    const int kchunks = K / (fmt == 2 ? 32 : 64);
    if (fmt == 2) e = launch_gemm<2>(ma, mb, ma, w, (int64_t)(M / BM) * (N / BN), kchunks, err, s, 0, withhold);
    else e = launch_gemm<1>(ma, mb, ma, w, (int64_t)(M / BM) * (N / BN), kchunks, err, s, 0, withhold);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    dev_free(Al, err, 256, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(EGS_ERR_CUDA, "egs_tc_gemm_test: %s", cudaGetErrorString(e));
    if (herr) return set_error(EGS_ERR_TIMEOUT, "egs_tc_gemm_test: a pipeline wait timed out");
    return EGS_OK;
}

extern "C" egs_status egs_tc_gemm_test(const void *A, const void *B, int32_t M, int32_t N, int32_t K, egs_precision p,
                                       float *C, void *stream)
{
    clear_error();
    return tc_gemm_test(A, B, M, N, K, p, C, -1, stream);
}

extern "C" egs_status egs_tc_gemm_test_withhold(const void *A, const void *B, int32_t M, int32_t N, int32_t K,
                                                egs_precision p, float *C, int64_t withhold_stage, void *stream)
{
    clear_error();
    if (withhold_stage < 0) return set_error(EGS_ERR_ARG, "egs_tc_gemm_test_withhold: withhold_stage must be >= 0");
    return tc_gemm_test(A, B, M, N, K, p, C, withhold_stage, stream);
}
