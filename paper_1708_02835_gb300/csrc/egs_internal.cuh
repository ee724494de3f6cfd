// Internal declarations shared by the CUDA translation units of libegs.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/egs.h"
#include "matern_params.h"

namespace egs {

// Device-side status of one evaluation.  fail_index is the first row whose
// Cholesky pivot was not positive (INT64_MAX = none).  result holds
// loglik, logdet, quad once the solve has finished.
struct DevStatus {
    unsigned long long fail_index;
    int timeout;
    int pad;
    double result[4];
};

constexpr unsigned long long kNoFail = 0xFFFFFFFFFFFFFFFFull;

__host__ __device__ inline int64_t tile_linear(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

// Geometry of a lower-tile matrix.
struct TileGeom {
    int64_t n;
    int b;
    int T;
    size_t tile_elems() const { return (size_t)b * (size_t)b; }
    size_t ntiles() const { return (size_t)T * (size_t)(T + 1) / 2; }
};

// Kernel classes for per-class device timing.
enum KernelClass { KC_GEN = 0, KC_POTRF, KC_TRSM, KC_UPDATE, KC_TRSV, KC_OTHER, KC_COUNT };

// Counts launches and, when enabled, brackets each launch with a CUDA event
// pair on the launching stream so the summed duration of each kernel class
// can be read after the stream has finished.
struct KernelTimer {
    bool on = false;
    int launches = 0;
    std::vector<cudaEvent_t> ev[KC_COUNT];
    void begin(int cls, cudaStream_t s)
    {
        if (!on) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev[cls].push_back(e);
    }
    void end(int cls, cudaStream_t s)
    {
        ++launches;
        if (!on) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev[cls].push_back(e);
    }
    // Summed milliseconds of a class (call after the stream has finished).
    double ms(int cls) const
    {
        double t = 0.0;
        for (size_t i = 0; i + 1 < ev[cls].size(); i += 2) {
            float x = 0.f;
            if (cudaEventElapsedTime(&x, ev[cls][i], ev[cls][i + 1]) == cudaSuccess) t += x;
        }
        return t;
    }
    ~KernelTimer()
    {
        for (auto &v : ev)
            for (auto e : v) cudaEventDestroy(e);
    }
};

#define EGS_LAUNCH(kt, cls, s, ...)      \
    do {                                 \
        if (kt) (kt)->begin((cls), (s)); \
        __VA_ARGS__;                     \
        if (kt) (kt)->end((cls), (s));   \
    } while (0)

// ---- launchers (stream-ordered, no synchronisation) ----
// Sigma(theta) into FP64 lower tiles.
cudaError_t launch_matern_tiles_f64(const double *X, const double *Y, const TileGeom &g,
                                    const egs_matern_params &P, double *tiles, cudaStream_t s,
                                    KernelTimer *kt = nullptr);

// Tile Cholesky in place (FP64).  Stops doing work once st->fail_index is set.
cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s,
                                   KernelTimer *kt = nullptr);

// Forward solve L y = z in place on zpad (T*b doubles, padded with zeros),
// with per-tile log-det / dot partials and the final assembly into st->result.
cudaError_t launch_trsv_tiles_f64(const double *tiles, const TileGeom &g, double *zpad, double *partials,
                                  DevStatus *st, cudaStream_t s, KernelTimer *kt = nullptr);

// Copy z (n doubles) into zpad (T*b doubles), zero padding.
cudaError_t launch_pad_vector(const double *z, int64_t n, double *zpad, int64_t npad, cudaStream_t s,
                              KernelTimer *kt = nullptr);

}  // namespace egs
