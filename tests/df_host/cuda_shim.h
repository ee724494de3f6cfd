// Host stand-ins for the CUDA intrinsics that matern_df.cuh uses, so that its
// double-float arithmetic can be checked on the CPU (compiled without FMA
// contraction; every operation rounds to nearest like its device
// counterpart).  rsqrtf is perturbed by a relative 2^-23, the size of the
// hardware approximation's error, so that the checks do not rely on an exact
// reciprocal square root.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__

static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __fsqrt_rn(float a) { return std::sqrt(a); }
static inline float __frsqrt_rn(float a) { return (float)(1.0 / std::sqrt((double)a)); }
static inline float rsqrtf(float a) { return (float)(1.0 / std::sqrt((double)a)) * (1.0f + 0x1p-23f); }
static inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
static inline unsigned __float_as_uint(float f) { unsigned i; std::memcpy(&i, &f, 4); return i; }
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline float __uint_as_float(unsigned i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline float __double2float_rn(double d) { return (float)d; }
static inline double __hiloint2double(int hi, int lo)
{
    const uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
}
struct float2 {
    float x, y;
};
struct float4 {
    float x, y, z, w;
};
