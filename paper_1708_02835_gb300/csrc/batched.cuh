// Per-problem device view shared by the batched drivers (batched.cu: one
// launch per step of every problem; batched_dag.cu: one persistent launch
// over the tile task graph of every problem).
#pragma once
#include "egs_internal.cuh"

namespace egs {

struct BatchProblem {
    const double *X, *Y, *z;
    int64_t n;
    int T, band;       // band >= T: every tile FP64 (the FP64 batch)
    double *tiles;     // FP64 tiles: T(T+1)/2 lower tiles, or the band tiles of a mixed problem
    float *f32;        // mixed: off-band FP32 tiles
    double *sig;       // mixed: dense FP64 copy of Sigma (lower tiles) for the refinement
    double *zpad;      // T*b: Z, then the forward solution y
    double *x, *d, *rows, *cols;  // mixed: T*b vectors
    double *partials;  // 2T
    DevStatus *st;
    const egs_matern_params *P;
    unsigned *cnt;     // persistent scheduler: T(T+1)/2 tile counters, then T vector-block counters
    double *mtab;      // EGS_MT_DOUBLES: the generator's local polynomials (general nu)
};

// The local polynomials of every general-nu problem of a batch: grid =
// (ceil(intervals / 8), nprob), one warp per sub-interval (batched.cu).
cudaError_t launch_batch_tables(const BatchProblem *probs, int nprob, cudaStream_t s);

}  // namespace egs
