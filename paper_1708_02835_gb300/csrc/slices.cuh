// Exact BF16 slicing of operand rows for the FP64-accurate tensor-core
// products of ozaki.cu (error-free splitting after Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59 (2012)).  A row x of length K <= 1024 with
// |x| < 2^e gets the scale s = 2^(e-7) and five slices q_1..q_5,
//   u = x / s (|u| < 128),  q_i = rint(r_i 2^{7(i-1)}) 2^{-7(i-1)},
//   r_1 = u,  r_{i+1} = r_i - q_i,
// every q_i an integer of at most 8 bits times a power of two (exact in
// BF16), so that x = s (q_1 + ... + q_5) up to s 2^-29.  Slice i of a row
// goes to dst[i * slice_stride + c].  One warp per row; lane owns the
// columns lane + 32 j.
#pragma once
#include <cuda_bf16.h>

namespace egs {

constexpr int kSlices = 5;

// FP64 rows (the band panel tiles and the dense test operands).
// Both return e (|x| < 2^e for every entry of the row; 0 for a zero row).
template <typename E>
__device__ __forceinline__ int slice_row(const E *__restrict__ src, int K, __nv_bfloat16 *__restrict__ dst,
                                         size_t slice_stride, double *scale)
{
    const int lane = threadIdx.x & 31;
    double x[32];
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int c = lane + 32 * j;
        x[j] = (c < K) ? (double)src[c] : 0.0;
        mx = fmax(mx, fabs(x[j]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    int e = 0;
    frexp(mx, &e);  // mx = f 2^e with f in [0.5, 1), so |x| < 2^e (mx = 0: e = 0)
    if (lane == 0) *scale = ldexp(1.0, e - 7);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int c = lane + 32 * j;
        if (c < K) {
            double u = ldexp(x[j], 7 - e);  // |u| < 128, exact
#pragma unroll
            for (int i = 0; i < kSlices; ++i) {
                const double q = ldexp(rint(ldexp(u, 7 * i)), -7 * i);  // exact in BF16
                dst[(size_t)i * slice_stride + c] = __float2bfloat16_rn((float)q);
                u -= q;  // exact
            }
        }
    }
    return e;
}

// FP32 rows (the off-band panel tiles): the same slices, computed in FP32 --
// every step is exact there too (u has at most 24 significant bits, and each
// q_i and remainder keeps a subset of them), so the FP64 pipe is not used.
__device__ __forceinline__ int slice_row_f32(const float *src, int K, __nv_bfloat16 *__restrict__ dst,
                                             size_t slice_stride, double *scale)
{
    const int lane = threadIdx.x & 31;
    float x[32];
    float mx = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int c = lane + 32 * j;
        x[j] = (c < K) ? src[c] : 0.0f;
        mx = fmaxf(mx, fabsf(x[j]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    int e = 0;
    frexpf(mx, &e);
    if (lane == 0) *scale = ldexp(1.0, e - 7);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int c = lane + 32 * j;
        if (c < K) {
            float u = ldexpf(x[j], 7 - e);
#pragma unroll
            for (int i = 0; i < kSlices; ++i) {
                const float p = (float)(1u << (7 * i)) , ip = 1.0f / p;  // powers of two: exact
                const float q = rintf(u * p) * ip;
                dst[(size_t)i * slice_stride + c] = __float2bfloat16_rn(q);
                u -= q;
            }
        }
    }
    return e;
}

}  // namespace egs
