// FP64-accurate products on the BF16 tensor cores by exact slicing (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)), used
// by the FP32 mixed mode for every update whose output is an FP64 band tile.
//
// Each operand row x (length K) is scaled by a power of two sigma = 2^e with
// |x| < sigma, u = x 128 / sigma, and cut into five slices (slices.cuh)
//   q_1 = rint(u),  q_i = rint((u - q_1 - ... - q_{i-1}) 2^{7(i-1)}) 2^{-7(i-1)},
// each an integer of at most 8 bits times a power of two, so exact in BF16;
// x = (sigma / 128) (q_1 + ... + q_5) up to 2^-36 sigma.  For a pair of rows
//   x . y = s_x s_y sum_{i,j} q_i(x) . q_j(y)        (s = sigma / 128)
// and the slice products are accumulated in FP32 on tcgen05 by level
// L = i + j (slices counted from 0), one accumulator per level:
//   acc_0 = q_1 . q_1                 integers, |acc_0| <= K 2^14 <= 2^23 (K <= 512)
//   acc_1 = q_1 . q_2 + q_2 . q_1     multiples of 2^-7, |acc_1| <= 2^23 units
//   acc_2, acc_3, acc_4               the 12 pairs with 2 <= i + j <= 4
// so acc_0 and acc_1 are exact in FP32 (the tensor core adds exact BF16
// products; every partial sum is a representable integer multiple of the
// level's unit below 2^24 units), and acc_2..acc_4 carry only rounding errors
// relative to their own magnitudes, 2^-14 and less of the result.  The
// epilogue forms acc_0 + acc_1 exactly as an FP32 pair (TwoSum), adds
// (acc_4 + acc_3) + acc_2 to the low part, scales by the power of two
// s_x s_y on the exponents and subtracts the two parts from the FP64 tile.
// Dropping the pairs with i + j > 4 leaves an error of about
// K 2^-35 s_x s_y 2^14, i.e. 35-bit products, which is the accuracy the band
// updates need (FP32-accurate products there are not enough; exact FP64 ones
// are).
//
// The 15 pair products of a K step are 5 MMAs: A slice i against the B
// slices 0 .. 4 - i, which lie back to back in shared memory and so form one
// operand of N = 32 (5 - i) rows; its D address is shifted by 32 i columns,
// so that the column block of B slice j lands in the accumulator of level
// i + j.  Each A slice is read from shared memory once per K step (instead of
// once per pair).
//
// Kernel: persistent, one CTA per SM, 192 threads.  Warp 0 (one lane) loads
// the five A slices (128 rows) and five B slices (32 rows) of a 64-element K
// chunk with TMA (128-byte swizzle) into a 2-stage ring; warp 1 (one lane)
// issues the 5 MMAs (M = 128, N = 160 .. 32, K = 16) of every K step into the
// five 32-column level accumulators, double-buffered across work items;
// warps 2-5 read the accumulators with tcgen05.ld and apply the FP64
// epilogue.
#include "egs_internal.cuh"
#include "slices.cuh"
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

namespace egs {

namespace {

constexpr int OS = kSlices;  // slices per operand
constexpr int OBM = 128, OBN = 32, OSTAGES = 2, OKC = 64;
constexpr int OA_SL = OBM * 128, OB_SL = OBN * 128;  // bytes of one slice box
constexpr int OSTAGE = OS * (OA_SL + OB_SL);
constexpr int OSMEM = OSTAGES * OSTAGE + 1024;
constexpr int ONUM_THREADS = 192;
constexpr int OLEV = OS;               // level accumulators (levels 0 .. 4)
constexpr int OBUF = OLEV * OBN;       // TMEM columns of one accumulator buffer
constexpr uint32_t OTMEM_COLS = 512;   // 2 buffers x 5 levels x 32 columns, rounded up

__device__ __forceinline__ bool ofailed(const DevStatus *st)
{
    return st && *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

// log2 of a power of two held in a double (the row scales).
__device__ __forceinline__ int pow2_exp(double p)
{
    return (int)((__double_as_longlong(p) >> 52) & 0x7FF) - 1023;
}

// x 2^esh as a double, exactly, built with integer operations (GB300 issues
// 2 FP64 operations per clock per SM, so the epilogue keeps conversions and
// scaling off the FP64 pipe).  FP32 zeros and subnormals (below 2^-126 of the
// accumulator unit, far under the result's last bit) give 0; inf / NaN stay
// inf / NaN.
__device__ __forceinline__ double f32_scaled(float x, int esh)
{
    const uint32_t u = __float_as_uint(x);
    const int ex = (int)((u >> 23) & 0xFFu);
    if (ex == 0) return 0.0;
    int e64 = (ex == 255) ? 2047 : ex - 127 + 1023 + esh;
    if (e64 <= 0) return 0.0;
    if (e64 > 2047) e64 = 2047;
    const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)e64 << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// Rows of a dense row-major FP64 matrix (rows x K) -> slices.
__global__ void __launch_bounds__(256) k_ozaki_slices_dense(const double *X, int rows, int K, __nv_bfloat16 *oz,
                                                            double *scale)
{
    const int r = (int)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    slice_row(X + (size_t)r * K, K, oz + (size_t)r * K, (size_t)rows * K, scale + r);
}

struct OzItem {
    int m, n;    // output tile
    int rb, cb;  // 128-row block, 32-column block
    int ya, yb;  // operand rows (within one slice) of the A and B boxes
};

// FP64-accurate outputs of step k not covered by the FP64 band x band
// update: tiles (m, n), n = col0 .. col0 + ncols - 1, m = n .. n + xband - 1
// < T, with m - k >= band (an FP32 panel operand).  C_mn -= P_m P_n^T in
// FP64; tiles with m - n >= band are FP32 and take the FP64 result rounded
// once.  With band_band set, the items are instead the band x band update
// itself (m - k < band: both operands FP64 band tiles).
struct OzBandWork {
    Tiles tl;
    int k, col0, xband, band_band;
    __device__ bool decode(int64_t item, OzItem &w) const
    {
        const int nrb = tl.b / OBM, ncb = tl.b / OBN, per = nrb * ncb;
        const int64_t t = item / per;
        const int blk = (int)(item % per);
        w.n = col0 + (int)(t / xband);
        w.m = w.n + (int)(t % xband);
        w.rb = blk / ncb;
        w.cb = blk % ncb;
        if (w.m >= tl.T || (w.m - k < tl.band) != (band_band != 0)) return false;
        if (w.m == w.n && w.cb * OBN > w.rb * OBM + OBM - 1) return false;  // strictly above the diagonal
        w.ya = (w.m - k - 1) * tl.b + w.rb * OBM;
        w.yb = (w.n - k - 1) * tl.b + w.cb * OBN;
        return true;
    }
    // C -= 2^(ea + eb_c) (hi_c + lo_c): two FP64 subtractions per entry
    __device__ void apply(const OzItem &w, int r, int ea, const int (&eb)[OBN], const float (&hi)[OBN],
                          const float (&lo)[OBN]) const
    {
        if (!tl.is64(w.m, w.n)) {
            float *C = tl.t32(w.m, w.n) + (size_t)(w.rb * OBM + r) * tl.b + w.cb * OBN;
            float4 c[OBN / 4];
#pragma unroll
            for (int i = 0; i < OBN / 4; ++i) c[i] = *reinterpret_cast<const float4 *>(C + 4 * i);
            float *cf = reinterpret_cast<float *>(c);
#pragma unroll
            for (int i = 0; i < OBN; ++i) {
                const int e = ea + eb[i];
                cf[i] = (float)(((double)cf[i] - f32_scaled(hi[i], e)) - f32_scaled(lo[i], e));
            }
#pragma unroll
            for (int i = 0; i < OBN / 4; ++i) *reinterpret_cast<float4 *>(C + 4 * i) = c[i];
            return;
        }
        double *C = tl.t64(w.m, w.n) + (size_t)(w.rb * OBM + r) * tl.b + w.cb * OBN;
        double2 c[OBN / 2];
#pragma unroll
        for (int i = 0; i < OBN / 2; ++i) c[i] = *reinterpret_cast<const double2 *>(C + 2 * i);
#pragma unroll
        for (int i = 0; i < OBN / 2; ++i) {
            const int e0 = ea + eb[2 * i], e1 = ea + eb[2 * i + 1];
            c[i].x = (c[i].x - f32_scaled(hi[2 * i], e0)) - f32_scaled(lo[2 * i], e0);
            c[i].y = (c[i].y - f32_scaled(hi[2 * i + 1], e1)) - f32_scaled(lo[2 * i + 1], e1);
        }
#pragma unroll
        for (int i = 0; i < OBN / 2; ++i) *reinterpret_cast<double2 *>(C + 2 * i) = c[i];
    }
};

// C = A B^T (A: M x K, B: N x K), used to test the pipeline.
struct OzDenseWork {
    double *C;
    int N, ncb;
    __device__ bool decode(int64_t item, OzItem &w) const
    {
        w.rb = (int)(item / ncb);
        w.cb = (int)(item % ncb);
        w.m = w.n = 0;
        w.ya = w.rb * OBM;
        w.yb = w.cb * OBN;
        return true;
    }
    __device__ void apply(const OzItem &w, int r, int ea, const int (&eb)[OBN], const float (&hi)[OBN],
                          const float (&lo)[OBN]) const
    {
        double *Cp = C + (size_t)(w.rb * OBM + r) * N + w.cb * OBN;
#pragma unroll
        for (int i = 0; i < OBN / 2; ++i) {
            const int e0 = ea + eb[2 * i], e1 = ea + eb[2 * i + 1];
            *reinterpret_cast<double2 *>(Cp + 2 * i) =
                make_double2(f32_scaled(hi[2 * i], e0) + f32_scaled(lo[2 * i], e0),
                             f32_scaled(hi[2 * i + 1], e1) + f32_scaled(lo[2 * i + 1], e1));
        }
    }
};

// mapA / mapB: 2-D maps over the slice arrays viewed as (OS * rows) x K BF16,
// boxes {64, 128} and {64, 32}; slice i of operand row y is map row
// i * RA + y (i * RB + y).
template <class Work>
__global__ void __launch_bounds__(ONUM_THREADS, 1)
k_tc_ozaki(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Work work,
           const double *__restrict__ scA, const double *__restrict__ scB, int RA, int RB, int64_t nitems, int kchunks,
           int *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[OSTAGES], empty[OSTAGES], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int last_chunk[OSTAGES];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
            last_chunk[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 4);
        }
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, OTMEM_COLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_tmap(&mapA);
            tc::prefetch_tmap(&mapB);
            int g = 0;
            for (int64_t item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
                OzItem wi;
                if (!work.decode(item, wi)) continue;
                for (int c = 0; c < kchunks; ++c, ++g) {
                    const int s = g % OSTAGES;
                    const uint32_t ph = (uint32_t)(g / OSTAGES) & 1u;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, &abort_flag)) break;
                    tc::mbar_arrive_expect_tx(&full[s], OSTAGE);
                    uint8_t *sa = smem + s * OSTAGE, *sb = sa + OS * OA_SL;
#pragma unroll
                    for (int i = 0; i < OS; ++i) {
                        tc::tma_load_2d(&mapA, &full[s], sa + i * OA_SL, c * OKC, i * RA + wi.ya);
                        tc::tma_load_2d(&mapB, &full[s], sb + i * OB_SL, c * OKC, i * RB + wi.yb);
                    }
                    last_chunk[s] = g;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // A slice i against B slices 0 .. 4 - i: N = 32 (5 - i)
            constexpr uint32_t idesc[OS] = {tc::idesc_f32acc(OBM, 5 * OBN, 1), tc::idesc_f32acc(OBM, 4 * OBN, 1),
                                            tc::idesc_f32acc(OBM, 3 * OBN, 1), tc::idesc_f32acc(OBM, 2 * OBN, 1),
                                            tc::idesc_f32acc(OBM, 1 * OBN, 1)};
            int g = 0, t = 0;
            for (int64_t item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
                OzItem wi;
                if (!work.decode(item, wi)) continue;
                const int buf = t & 1;
                const uint32_t use = (uint32_t)(t >> 1);
                if (!tc::mbar_wait(&tempty[buf], (use & 1u) ^ 1u, &abort_flag)) break;
                tc::tc_fence_after();
                const uint32_t d = tbase + (uint32_t)buf * OBUF;
                for (int c = 0; c < kchunks; ++c, ++g) {
                    const int s = g % OSTAGES;
                    const uint32_t ph = (uint32_t)(g / OSTAGES) & 1u;
                    if (!tc::mbar_wait(&full[s], ph, &abort_flag)) break;
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(smem + s * OSTAGE);
                    const uint32_t b0 = a0 + OS * OA_SL;
#pragma unroll
                    for (int j = 0; j < OKC / 16; ++j) {
                        const uint64_t bd = tc::desc_sw128(b0 + 32 * j);
#pragma unroll
                        for (int i = 0; i < OS; ++i) {
                            // the i = 0 MMA of the first K step covers all five
                            // level blocks and so initialises them
                            const uint64_t ad = tc::desc_sw128(a0 + i * OA_SL + 32 * j);
                            tc::mma_f16(d + (uint32_t)(i * OBN), ad, bd, idesc[i], ((c | j) != 0 || i != 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&tfull[buf]);
                ++t;
            }
        }
    } else {
        // warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. output
        // rows 32 (w % 4) + lane of the 128-row block
        const int q = warp & 3;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int t = 0;
        for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
            OzItem wi;
            if (!work.decode(item, wi)) continue;
            const int buf = t & 1;
            const uint32_t use = (uint32_t)(t >> 1);
            const bool ok = tc::mbar_wait(&tfull[buf], use & 1u, &abort_flag);
            tc::tc_fence_after();
            if (!__all_sync(0xffffffffu, ok && !abort_flag)) break;
            const uint32_t d = tbase + (uint32_t)buf * OBUF + lane_base;
            float a0v[32], a1v[32], a2v[32], tv[32];
            tc::tmem_ld32(d + 4 * OBN, a2v);
            tc::tmem_ld32(d + 3 * OBN, tv);
#pragma unroll
            for (int c = 0; c < OBN; ++c) a2v[c] += tv[c];
            tc::tmem_ld32(d + 2 * OBN, tv);
#pragma unroll
            for (int c = 0; c < OBN; ++c) a2v[c] += tv[c];
            tc::tmem_ld32(d, a0v);
            tc::tmem_ld32(d + OBN, a1v);
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);  // the accumulators are in registers now
            // (acc_0 + acc_1) exactly as hi + e (Knuth's TwoSum in FP32), then
            // lo = e + ((acc_4 + acc_3) + acc_2) (rounded 2^-24 below acc_2,
            // itself 2^-14 below the result); the row scales are powers of
            // two, applied to the exponents
            const int r = q * 32 + lane;
            const int ea = pow2_exp(scA[wi.ya + r]);
            int eb[OBN];
#pragma unroll
            for (int c = 0; c < OBN; ++c) {
                eb[c] = pow2_exp(__ldg(scB + wi.yb + c));
                const float x = a0v[c], y = a1v[c];
                const float s = x + y;
                const float bv = s - x;
                const float e = (x - (s - bv)) + (y - bv);
                a0v[c] = s;
                a1v[c] = e + a2v[c];
            }
            work.apply(wi, r, ea, eb, a0v, a1v);
            ++t;
        }
    }
    __syncwarp();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s)
            if (last_chunk[s] >= 0) {
                volatile int dummy = 0;
                tc::mbar_wait(&full[s], (uint32_t)(last_chunk[s] / OSTAGES) & 1u, &dummy);
            }
        atomicExch(err, 1);
    }
    tc::tc_fence_after();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, OTMEM_COLS);
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn()
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

// 2-D map over OS * rows rows of K BF16, box {64, box_rows}, 128-byte swizzle.
cudaError_t make_slice_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t K, uint32_t box_rows)
{
    auto fn = oz_encode_fn();
    if (!fn) return cudaErrorNotSupported;
    cuuint64_t dims[2] = {K, (cuuint64_t)OS * rows};
    cuuint64_t strides[1] = {K * 2};
    cuuint32_t box[2] = {(cuuint32_t)OKC, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int oz_num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    }
    return sms;
}

template <class Work>
cudaError_t launch_ozaki(const CUtensorMap &ma, const CUtensorMap &mb, const Work &w, const double *scA,
                         const double *scB, int RA, int RB, int64_t items, int kchunks, int *err, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_ozaki<Work>, cudaFuncAttributeMaxDynamicSharedMemorySize, OSMEM);
    if (e != cudaSuccess) return e;
    const int64_t grid = items < oz_num_sms() ? items : oz_num_sms();
    k_tc_ozaki<Work><<<(unsigned)grid, ONUM_THREADS, OSMEM, s>>>(ma, mb, w, scA, scB, RA, RB, items, kchunks, err);
    return cudaGetLastError();
}

}  // namespace

size_t ozaki_slices_bytes(int b, int T)
{
    const size_t R = (size_t)(T > 1 ? T - 1 : 1) * (size_t)b;
    return (size_t)OS * R * (size_t)b * 2;
}

cudaError_t make_ozaki_maps(const void *oz, int b, int T, CUtensorMap *mapA, CUtensorMap *mapB)
{
    const uint64_t R = (uint64_t)(T > 1 ? T - 1 : 1) * (uint64_t)b;
    cudaError_t e = make_slice_map(mapA, oz, R, (uint64_t)b, OBM);
    if (e == cudaSuccess) e = make_slice_map(mapB, oz, R, (uint64_t)b, OBN);
    return e;
}

cudaError_t launch_band_out_ozaki(const CUtensorMap &mapA, const CUtensorMap &mapB, const Tiles &tl, int xband, int k,
                                  int col0, int ncols, const double *scale, int *err, cudaStream_t s, KernelTimer *kt)
{
    if (ncols <= 0) return cudaSuccess;
    if (xband < tl.band) xband = tl.band;
    const int64_t per = (int64_t)(tl.b / OBM) * (tl.b / OBN);
    const int64_t items = (int64_t)ncols * xband * per;
    const int R = (tl.T - 1) * tl.b;
    OzBandWork w{tl, k, col0, xband, 0};
    cudaError_t e;
    if (kt) kt->begin(KC_UPDATE64, s);
    e = launch_ozaki(mapA, mapB, w, scale, scale, R, R, items, tl.b / OKC, err, s);
    if (kt) kt->end(KC_UPDATE64, s);
    return e;
}

cudaError_t launch_band_band_ozaki(const CUtensorMap &mapA, const CUtensorMap &mapB, const Tiles &tl, int k, int nb,
                                   const double *scale, int *err, cudaStream_t s, KernelTimer *kt)
{
    if (nb <= 0) return cudaSuccess;
    const int64_t per = (int64_t)(tl.b / OBM) * (tl.b / OBN);
    const int64_t items = (int64_t)nb * nb * per;
    const int R = (tl.T - 1) * tl.b;
    OzBandWork w{tl, k, k + 1, nb, 1};
    cudaError_t e;
    if (kt) kt->begin(KC_UPDATE64, s);
    e = launch_ozaki(mapA, mapB, w, scale, scale, R, R, items, tl.b / OKC, err, s);
    if (kt) kt->end(KC_UPDATE64, s);
    return e;
}

}  // namespace egs

using namespace egs;

extern "C" egs_status egs_ozaki_gemm_test(const double *A, const double *B, int32_t M, int32_t N, int32_t K, double *C,
                                          void *stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || M % OBM || N % OBN || K % OKC || K > 512)
        return set_error(EGS_ERR_ARG, "egs_ozaki_gemm_test: M %% 128, N %% 32, K %% 64 must be 0 and K <= 512");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sa = (size_t)OS * M * K * 2, sb = (size_t)OS * N * K * 2;
    char *ws = nullptr;
    const size_t bytes = sa + sb + (size_t)(M + N) * 8 + 256;
    const Allocator Al = current_allocator();
    cudaError_t e = dev_alloc(Al, (void **)&ws, bytes, s);
    if (e != cudaSuccess) return set_error(EGS_ERR_OOM, "egs_ozaki_gemm_test: workspace");
    __nv_bfloat16 *oa = (__nv_bfloat16 *)ws, *ob = (__nv_bfloat16 *)(ws + sa);
    double *sca = (double *)(ws + sa + sb), *scb = sca + M;
    int *err = (int *)(scb + N);
    CUtensorMap ma, mb;
    e = make_slice_map(&ma, oa, (uint64_t)M, (uint64_t)K, OBM);
    if (e == cudaSuccess) e = make_slice_map(&mb, ob, (uint64_t)N, (uint64_t)K, OBN);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_ozaki_slices_dense<<<(unsigned)((M + 7) / 8), 256, 0, s>>>(A, M, K, oa, sca);
        k_ozaki_slices_dense<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(B, N, K, ob, scb);
        e = cudaGetLastError();
    }
    OzDenseWork w{C, N, N / OBN};
    if (e == cudaSuccess) e = launch_ozaki(ma, mb, w, sca, scb, M, N, (int64_t)(M / OBM) * (N / OBN), K / OKC, err, s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    dev_free(Al, ws, bytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(EGS_ERR_CUDA, "egs_ozaki_gemm_test: %s", cudaGetErrorString(e));
    if (herr) return set_error(EGS_ERR_TIMEOUT, "egs_ozaki_gemm_test: a pipeline wait timed out");
    return EGS_OK;
}
