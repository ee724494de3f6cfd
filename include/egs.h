/*
 * egs.h - C ABI of the GB300 exact Gaussian log-likelihood library (libegs.so).
 *
 * The library evaluates Eq. 1 of Abdulah et al., "ExaGeoStat: A High
 * Performance Unified Software for Geostatistics on Manycore Systems"
 * (arXiv:1708.02835), Section 2:
 *
 *     l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 Z^T Sigma(theta)^-1 Z
 *
 * with Sigma_ij = C(||s_i - s_j||; theta) from the Matern covariance, Eq. 2
 * (Section 2.2):
 *
 *     C(r; theta) = theta1 / (2^(theta3 - 1) Gamma(theta3)) (r/theta2)^theta3 K_theta3(r/theta2)
 *
 * following Algorithm 2 (Section 6.5): generate Sigma, factor Sigma = L L^T by
 * tile Cholesky, solve L y = Z, reduce log|Sigma| = 2 sum_i log L_ii and
 * y^T y, and assemble l.  Every step runs in the library's own sm_103a CUDA
 * kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Locations are passed as one array of 2n doubles: x[0..n) then y[0..n).
 * - theta is a host array of 3 doubles (theta1 variance, theta2 range,
 *   theta3 smoothness); each must be finite and > 0 (Section 2.2), otherwise
 *   EGS_ERR_ARG.
 * - n >= 1.  tile (the Cholesky tile size b) is a multiple of 64 in [64, 1024];
 *   0 selects the library default for n and precision.
 * - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Device buffers passed in are borrowed for the duration of the
 *   call; the library keeps no pointer to them afterwards.
 * - Errors are return codes; nothing aborts, traps or prints.  A thread-local
 *   message is available from egs_last_error().  When the matrix is not
 *   positive definite the call returns EGS_ERR_NOT_PD, the log-likelihood is
 *   NaN and egs_info.fail_index holds the first failing row.
 *
 * Tile layout ("lower tiles")
 * ---------------------------
 * T = ceil(n / b).  Only tiles (i, j) with i >= j are stored, tile (i, j) at
 * position i (i + 1) / 2 + j, each tile b x b contiguous and row-major
 * (element (r, c) at r * b + c).  Rows and columns at or beyond n are padding:
 * zero, except padded diagonal entries, which are one, so the padded matrix
 * is positive definite with the same log-determinant and quadratic form.
 * In EGS_FP64 every tile is double.  (Mixed-precision layouts are described
 * at egs_tiles_bytes.)
 */
#ifndef EGS_H
#define EGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EGS_OK = 0,
    EGS_ERR_ARG = 1,           /* invalid argument (sizes, theta, pointers) */
    EGS_ERR_NOT_PD = 2,        /* Cholesky met a pivot <= 0 (or NaN) */
    EGS_ERR_OOM = 3,           /* device allocation failed or budget exceeded */
    EGS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    EGS_ERR_TIMEOUT = 5,       /* a bounded wait expired */
    EGS_ERR_BUSY = 6,          /* resource busy (serving: queue full) */
    EGS_ERR_UNIMPLEMENTED = 7, /* feature not built */
    EGS_ERR_INACCURATE = 8     /* mixed precision only: the FP64 refinement step
                                  changed the quadratic form by more than 1e-5
                                  (EGS_MIX_FP32; the l it passes is then within
                                  a few 1e-5 of FP64) or 1e-3 (TF32 / BF16: a
                                  guard against gross errors) relative, i.e. the
                                  mixed factor is too inexact for Sigma(theta)
                                  (condition number near 1/eps of the off-band
                                  precision); the value is still in
                                  egs_info.loglik -- evaluate this theta in
                                  EGS_FP64 */
} egs_status;

typedef enum {
    EGS_FP64 = 0,     /* everything in double */
    EGS_MIX_FP32 = 1, /* FP64 band; off-band tiles FP32; updates of band tiles
                         (and of the tiles within egs_opts.xband of the
                         diagonal) FP64-accurate (DFMA, or exact BF16 slice
                         products on tcgen05), of the other off-band tiles on
                         tcgen05 as split FP16 (lo hi' + hi lo' + hi hi' of
                         row-scaled FP16 halves, FP32-accurate products); the
                         off-band TRSM as the split-TF32 product with the
                         FP64 inverse of the diagonal tile */
    EGS_MIX_TF32 = 2, /* FP64 band; off-band tiles FP32, updates on tcgen05 TF32 */
    EGS_MIX_BF16 = 3  /* FP64 band; off-band operands BF16, FP32 accumulation */
} egs_precision;

/* Per-call diagnostics (all fields written by the call when non-NULL). */
typedef struct {
    double loglik;        /* l(theta), NaN on failure */
    double logdet;        /* log|Sigma| = 2 sum_i log L_ii */
    double quad;          /* Z^T Sigma^-1 Z */
    int64_t fail_index;   /* first row whose pivot failed, or -1 */
    int64_t fail_tile;    /* fail_index / tile, or -1 */
    int32_t tile;         /* tile size used */
    int32_t band;         /* FP64 band width in tiles (mixed modes) */
    int32_t launches;     /* kernels this call launched */
    int32_t refine_steps; /* FP64 refinement steps taken (mixed modes) */
    double quad_unrefined;/* mixed modes: Z^T Sigma^-1 Z before refinement */
    /* Device times in ms (CUDA events on the call's stream; zero unless
     * egs_opts.timing is set).  timing = 1: per phase; timing = 2: also the
     * summed duration of each kernel class (one event pair per launch). */
    double ms_generate;   /* Sigma generation */
    double ms_factor;     /* tile Cholesky */
    double ms_solve;      /* solve, refinement and reductions */
    double ms_total;      /* whole evaluation */
    double ms_potrf;      /* timing = 2: diagonal-tile POTRF kernels */
    double ms_trsm;       /* timing = 2: panel TRSM kernels */
    double ms_update;     /* timing = 2: SYRK/GEMM trailing-update kernels */
    double ms_trsv;       /* timing = 2: solve kernels */
    double ms_update_f64; /* timing = 2, mixed precision: the FP64 update launches
                             (band x band, and in EGS_MIX_FP32 every band output);
                             ms_update then counts only the tensor-core update */
} egs_info;

/* Optional knobs for egs_loglik_ex.  Zero-initialise for defaults. */
typedef struct {
    int32_t tile;          /* 0 = default */
    int32_t band;          /* FP64 band width in tiles for mixed modes; 0 = 2 */
    int32_t refine;        /* mixed modes: FP64 refinement steps (0 = default 1, -1 = none) */
    int32_t timing;        /* nonzero: record per-phase CUDA events into egs_info;
                              >= 3: also keep a per-launch trace (egs_trace_last) */
    void *workspace;       /* caller-owned device workspace, or NULL (library allocates) */
    size_t workspace_bytes;
    int32_t distance;      /* 0: Euclidean on (x, y); 1: great-circle distance on
                              (longitude, latitude) in degrees by the haversine
                              formula (Section 7.4) on a sphere of 6371 km, so
                              theta2 is in km */
    int32_t xband;         /* EGS_MIX_FP32 only: tiles with i - j < xband receive
                              FP64-accurate updates (exact BF16 slice products)
                              although those with i - j >= band are stored in
                              FP32; 0 = band (must be >= band otherwise) */
} egs_opts;

/* One kernel launch of a traced evaluation (egs_opts.timing >= 3). */
typedef struct {
    int32_t kclass;   /* 0 Sigma generation, 1 diagonal POTRF, 2 panel TRSM (and the
                         operand preparation of the mixed modes), 3 trailing update
                         (tensor-core in the mixed modes), 4 solve, 5 other
                         (refinement, reductions), 6 FP64-accurate band update */
    int32_t step;     /* factorisation step k of the launch, -1 outside the factorisation */
    int32_t stream;   /* 0: the call's stream; 1: the library's lookahead stream */
    int32_t reserved;
    double start_ms;  /* CUDA-event times relative to the start of Sigma generation */
    double end_ms;
} egs_trace_rec;

/* Copies the calling thread's trace of its last egs_loglik_ex call made with
 * timing >= 3 into out[0 .. min(cap, *count) - 1], in enqueue order, and sets
 * *count to the number of records (call with cap = 0 to size the buffer).
 * Events bracket each launch on its stream, so a record includes any time the
 * launch waited for SMs.  EGS_ERR_ARG if count is NULL or out is NULL with
 * cap > 0.  Host-only; no GPU work. */
egs_status egs_trace_last(egs_trace_rec *out, int64_t cap, int64_t *count);

/*
 * egs_set_allocator - the device memory of the library's calls (per-call
 * workspaces, serving slots and fields, batch plans) from the caller's
 * allocator, for example a framework's caching allocator, instead of
 * cudaMallocAsync / cudaFreeAsync on the call's stream.  The paper has no
 * counterpart: this is the boundary's memory-management convention.
 *   alloc(bytes, stream, ctx)   returns device memory of at least bytes
 *                               bytes, usable in stream order on stream
 *                               (a cudaStream_t), aligned to 256 bytes; NULL
 *                               when it cannot (the call then fails with
 *                               EGS_ERR_OOM)
 *   free(ptr, bytes, stream, ctx)  returns it; work already enqueued on
 *                               stream may still use ptr, so the allocator
 *                               must not hand it out to another stream
 *                               before that work has finished
 * Both NULL restores cudaMallocAsync / cudaFreeAsync; one NULL is
 * EGS_ERR_ARG.  Memory is always returned to the allocator that provided it,
 * also when the allocator is replaced in the meantime.  The library may call
 * the hooks from its serving thread, with its internal locks held: a hook
 * must not call back into the library.  A server or batch keeps the
 * allocator that was set when it was created.  Process-wide; host-only, no
 * GPU work.
 */
typedef void *(*egs_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*egs_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
egs_status egs_set_allocator(egs_alloc_fn alloc, egs_free_fn free_fn, void *ctx);

/* Message describing the last error on the calling thread ("" if none). */
const char *egs_last_error(void);

/* Library version string. */
const char *egs_version(void);

/* Default tile size for n in the given precision. */
int32_t egs_default_tile(int64_t n, egs_precision p);

/* Bytes of the lower-tile matrix for (n, tile, p, band).  EGS_FP64: all
 * T (T + 1) / 2 tiles are double.  Mixed precisions (band <= 0 means 2; when
 * T <= band every tile is double): the band tiles (i - j < band) are double,
 * stored band by band at position i * band + (i - j), and the other tiles are
 * float at position (i - band)(i - band + 1) / 2 + j of a second array that
 * follows; the total of both is returned.  Returns 0 for invalid arguments. */
size_t egs_tiles_bytes(int64_t n, int32_t tile, egs_precision p, int32_t band);

/* Bytes of device workspace egs_loglik_ex needs for (n, tile, p, band),
 * including the tile matrix.  Returns 0 for invalid arguments. */
size_t egs_loglik_workspace_bytes(int64_t n, int32_t tile, egs_precision p, int32_t band);

/*
 * egs_matern_tiles - generate Sigma(theta) (Eq. 2; Algorithm 2, genCovMatrix)
 * into the lower-tile layout of precision p (egs_tiles_bytes): EGS_FP64 every
 * tile double; the mixed precisions the band tiles (i - j < band, band <= 0
 * meaning 2) as doubles and the other tiles rounded to float in the second
 * array (all double when T <= band).  FP64 tiles are computed in FP64; the
 * float tiles of a mixed layout, under the Euclidean distance, in double-float
 * arithmetic (float pairs, about 1e-14 relative) and rounded once.
 *   locs   device, 2n doubles (x then y)
 *   tiles  device, egs_tiles_bytes(n, tile, p, band) bytes, written
 * Entries with r = 0 take the limit C(0) = theta1.  Asynchronous on stream.
 * EGS_ERR_ARG if locs or tiles is not device memory.
 */
egs_status egs_matern_tiles(const double *locs, int64_t n, const double theta[3], int32_t tile,
                            egs_precision p, int32_t band, void *tiles, void *stream);

/*
 * egs_potrf_tiles - tile Cholesky Sigma = L L^T in place (Algorithm 2,
 * dpotrf; the right-looking tile algorithm of Section 5.2: POTRF on the
 * diagonal tile, TRSM on the panel, SYRK/GEMM on the trailing tiles).
 *   tiles       device, lower tiles of Sigma in EGS_FP64 layout; on return L
 *   fail_index  host; first failing row or -1.  The call synchronises stream.
 * EGS_ERR_ARG if tiles is not device memory.
 */
egs_status egs_potrf_tiles(void *tiles, int64_t n, int32_t tile, int64_t *fail_index, void *stream);

/*
 * egs_trsv_tiles - forward solve L y = Z (Algorithm 2, dtrsm; Section 6.5
 * states it as L Z_new = Z_old) with the log-determinant (2 sum_i log L_ii,
 * Section 6.1) and the dot product y^T y (Algorithm 2, computeDotProduct).
 *   tiles  device, L in EGS_FP64 lower-tile layout
 *   z      device, n doubles;  y  device, n doubles (may alias z)
 *   logdet, quad  host; the call synchronises stream.
 * EGS_ERR_ARG if tiles, z or y is not device memory.
 */
egs_status egs_trsv_tiles(const void *tiles, int64_t n, int32_t tile, const double *z, double *y,
                          double *logdet, double *quad, void *stream);

/*
 * egs_trsv_tiles_noalloc - egs_trsv_tiles for callers that cannot allocate
 * device memory during the call (for example an application whose own
 * memory manager has reserved the whole device, or a latency-sensitive loop
 * that cannot afford the device-wide synchronisation cudaFree implies).  The
 * paper has no counterpart; it is a deployment variant of the solve above.
 * Same arguments, results and errors as egs_trsv_tiles, but the scratch (the
 * padded solution vector, the per-tile partial sums and the status word)
 * lives in one fixed device array inside the library, about 1.1 MB, that
 * every GPU which loads the library keeps until the process exits; nothing is
 * allocated or freed.  Limits: ceil(n / tile) * tile <= 131072 and
 * ceil(n / tile) <= 2048, otherwise EGS_ERR_ARG with a message (use
 * egs_trsv_tiles).  The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first call
 * before any stream capture.  After cudaDeviceReset the next call on that
 * device looks the address up again (the module is reloaded), so that call
 * too should come before any capture.  z, y and tiles must be device memory
 * (EGS_ERR_ARG otherwise).  All calls share the one array and it keeps the
 * last call's contents: calls that overlap on the GPU (for example on two
 * streams) race and must be serialised by the caller.  Synchronises stream.
 */
egs_status egs_trsv_tiles_noalloc(const void *tiles, int64_t n, int32_t tile, const double *z, double *y,
                                  double *logdet, double *quad, void *stream);

/*
 * egs_simulate - synthetic measurements, Algorithm 1 (Section 6.4): generate
 * Sigma(theta) at the locations, factor Sigma = L L^T in FP64 (dpotrf) and
 * form Z = L e (dtrmm) for a caller-supplied e (normally e ~ N(0, I)).
 *   locs  2n doubles (x then y), device or host;  e  n doubles, device or host
 *   z     device, n doubles, written.  tile 0 = default.
 * EGS_ERR_NOT_PD if Sigma(theta) is not positive definite in FP64.
 * Synchronises stream.
 */
egs_status egs_simulate(const double *locs, const double *e, const double theta[3], int64_t n, int32_t tile, double *z,
                        void *stream);

/*
 * egs_loglik - one evaluation of Eq. 1 (Algorithm 2) at theta.
 *   locs  2n doubles (x then y), device or host memory
 *   z     n doubles, device or host memory
 *   out_loglik  host; info nullable.
 * Host inputs are copied to the device inside the call.  Workspace comes
 * from a stream-ordered device pool.  Synchronises stream before returning.
 */
egs_status egs_loglik(const double *locs, const double *z, const double theta[3], int64_t n,
                      egs_precision p, double *out_loglik, egs_info *info, void *stream);

/* egs_loglik with options (tile, band, refinement, caller workspace).
 * Mixed precisions: each refinement step forms the FP64 residual
 * Z - Sigma x with every entry of Sigma(theta) regenerated tile by tile (no
 * copy of Sigma is stored; Euclidean distance: double-float entries within
 * about 1e-14 relative, great-circle distance: the FP64 evaluation).  With
 * refine >= 1 the call returns EGS_ERR_INACCURATE (out_loglik untouched,
 * info filled) when the first step does not contract. */
egs_status egs_loglik_ex(const double *locs, const double *z, const double theta[3], int64_t n,
                         egs_precision p, const egs_opts *opts, double *out_loglik, egs_info *info,
                         void *stream);

/*
 * Batched evaluation (independent problems: uneven n, own theta each).
 *
 * Each problem is Eq. 1 evaluated by Algorithm 2 exactly as egs_loglik does
 * in EGS_FP64.  EGS_FP64 batches with tile <= 256 run as ONE persistent
 * kernel launch: the tile tasks of every problem (Matern tiles, the POTRF /
 * TRSM / SYRK-GEMM tasks of the tile Cholesky of Section 5.2 -- the DAG of
 * its tile algorithm -- and the forward-solve tasks) form one list in a
 * dependency order checked when the plan is made, and each CTA claims the
 * next task and waits on per-tile device counters until its inputs are final
 * (every wait bounded: EGS_ERR_TIMEOUT if one runs out).  Every l is bitwise
 * equal to egs_loglik_ex's with the same tile.  Other batches (EGS_MIX_FP32,
 * or tiles above 256) run as step-synchronous launches, each covering one
 * step of every problem.  Either way the run is captured into a CUDA graph on
 * the first egs_batch_run and replayed afterwards.
 *
 * egs_batch_create  plan for nprob problems of sizes n[0..nprob) with one tile
 *                   size for the batch (0 = the tile egs_batch_autotune found
 *                   for this size class and precision, else 64 up to n = 2048
 *                   and 128 above); owns all device memory of the batch
 *                   (egs_batch_workspace_bytes).
 * egs_batch_run     locs[i] (2 n[i] doubles, x then y) and z[i] (n[i]
 *                   doubles), device or host memory; theta: nprob x 3 host
 *                   doubles.  out[i] = l_i (NaN if problem i is not positive
 *                   definite), per_status[i] its status (both nullable).
 *                   Synchronises stream.  Returns EGS_ERR_NOT_PD if any
 *                   problem failed (the others are still valid).
 * egs_loglik_batched  create + run + destroy in one call.
 * Batches are EGS_FP64 or EGS_MIX_FP32: an FP64 band of 2 tiles, FP32
 * off-band tiles updated in FP32 on the CUDA cores, FP64 products for every
 * band tile, one FP64 refinement step against an FP64 copy of Sigma (a
 * problem of at most 2 tiles is all FP64); per_status[i] is
 * EGS_ERR_INACCURATE when that step changes Z^T x by more than 1e-5 relative.
 */
typedef struct egs_batch egs_batch;
egs_status egs_batch_create(int32_t nprob, const int64_t *n, int32_t tile, egs_precision p, egs_batch **out);
egs_status egs_batch_run(egs_batch *batch, const double *const *locs, const double *const *z, const double *theta,
                         double *out, egs_status *per_status, void *stream);
egs_status egs_batch_destroy(egs_batch *batch);
int32_t egs_batch_launches(const egs_batch *batch);     /* kernels per run (in the graph) */
int32_t egs_batch_tile(const egs_batch *batch);
size_t egs_batch_workspace_bytes(const egs_batch *batch);
egs_status egs_loglik_batched(int32_t nprob, const int64_t *n, const double *const *locs, const double *const *z,
                              const double *theta, egs_precision p, double *out, egs_status *per_status,
                              void *stream);

/*
 * egs_batch_autotune - the tile autotuner of the batched scheduler: builds a
 * batch of these problems with each candidate tile (64, 128, 256), runs it
 * twice on the caller's inputs (same arguments as egs_batch_run) and times
 * the second run with CUDA events on stream; the fastest tile is stored in
 * the library's table under (ceil(log2(largest n)), p), where
 * egs_batch_create with tile = 0 finds it for later batches of that size
 * class.  *best_tile (nullable) receives it, ms[0..2] (nullable) the three
 * run times.  Allocates and synchronises; problems that are not positive
 * definite do not stop the tuning.
 */
egs_status egs_batch_autotune(int32_t nprob, const int64_t *n, const double *const *locs, const double *const *z,
                              const double *theta, egs_precision p, int32_t *best_tile, double *ms, void *stream);
/* Tile stored by egs_batch_autotune for batches whose largest n is nmax, or 0. */
int32_t egs_batch_tuned_tile(int64_t nmax, egs_precision p);

/* Tasks in the persistent launch of a batch (0 for a step-synchronous batch). */
int64_t egs_batch_tasks(const egs_batch *batch);
/*
 * egs_batch_set_wait_limit - failure detection of the persistent launch:
 * every dependency wait gives up after limit_ns nanoseconds (default 10 s)
 * and the run returns EGS_ERR_TIMEOUT (all per_status EGS_ERR_TIMEOUT, out
 * NaN) with the batch still usable.  withhold_task in [0, egs_batch_tasks)
 * makes the launch never signal that task's completion, so that the waits
 * on it run out (for tests of this path); -1 signals every task.  Applies to
 * the following runs.  EGS_ERR_UNIMPLEMENTED for a step-synchronous batch.
 */
egs_status egs_batch_set_wait_limit(egs_batch *batch, int64_t limit_ns, int64_t withhold_task);

/*
 * egs_predict - kriging prediction, Eq. 5 by Algorithm 3 (Section 6.6): with
 * zero means, Z_1 = Sigma_12 Sigma_22^-1 Z_2 for m new locations given n
 * observed ones and their measurements Z_2.  Sigma_22 is factored as in one
 * egs_loglik_ex evaluation with the same precision and options (FP64: tile
 * Cholesky, forward and backward solves; mixed: the refined x = Sigma_22^-1
 * Z_2 of the evaluation); Sigma_12 is formed on the fly and never stored.
 *   locs_obs  2n doubles (x then y), z_obs n doubles;  locs_new 2m doubles
 *   z_new     m doubles, written;  all device or host memory
 *   info      (nullable) the evaluation's loglik / logdet / quad at theta
 * EGS_ERR_NOT_PD / EGS_ERR_INACCURATE as egs_loglik_ex.  Synchronises stream.
 */
egs_status egs_predict(const double *locs_obs, const double *z_obs, int64_t n, const double *locs_new, int64_t m,
                       const double theta[3], egs_precision p, const egs_opts *opts, double *z_new, egs_info *info,
                       void *stream);

/*
 * egs_loglik_ind - the independent-blocks (IND) approximation of Section 6.8:
 * every tile outside the diagonal super tiles (super_tiles x super_tiles
 * tiles of tile x tile) is set to zero, so Sigma is block diagonal over
 * consecutive runs of super_tiles * tile locations (the last run holds the
 * rest), and l_IND = sum over the blocks of Eq. 1 on each block's locations
 * and measurements.  FP64; the blocks run as one batch of the batched
 * scheduler (one CUDA graph).  Sums over the blocks are in block order.
 *   locs  2n doubles (x then y), device or host;  z  n doubles, device or host
 *   tile  0 = 128;  super_tiles >= 1 (super_tiles * tile >= n gives exact l)
 *   info  loglik, logdet, quad summed over the blocks; band = super_tiles
 * EGS_ERR_NOT_PD (fail_index = global row) if a block is not positive
 * definite.  Synchronises stream; allocates its workspace per call.
 */
egs_status egs_loglik_ind(const double *locs, const double *z, const double theta[3], int64_t n, int32_t tile,
                          int32_t super_tiles, double *out_loglik, egs_info *info, void *stream);

/*
 * Serving loop: likelihood requests from concurrent optimisers.
 *
 * Fields (locations + measurements) are copied to the device once and stay
 * resident.  Requests (field, theta, precision) enter a FIFO queue; a
 * scheduler thread admits the head request as soon as an execution slot is
 * free and its workspace fits in the HBM budget (resident fields plus
 * workspaces in flight <= hbm_budget_bytes), and enqueues it on the slot's own
 * stream, so requests that arrive while others run overlap with them on the
 * GPU.  Each evaluation is exactly egs_loglik's (deterministic kernels), so a
 * result is the same alone and in the mix.  Latency is measured from submit
 * to completion on the host clock.
 *   egs_serve_create    config: budget in bytes, 1..64 slots, tile/band for
 *                       the evaluations (0 = defaults).
 *   egs_serve_add_field locs (2n doubles, x then y) and z (n doubles), host or
 *                       device; the server copies them.  EGS_ERR_OOM if the
 *                       field does not fit in the budget.
 *   egs_serve_submit    non-blocking; returns a ticket.
 *   egs_serve_wait      timeout_ms < 0 waits forever; EGS_ERR_TIMEOUT if not
 *                       done in time (the request stays queued / running);
 *                       EGS_ERR_NOT_PD etc. from the evaluation; EGS_ERR_OOM
 *                       if the request's workspace does not fit in the budget
 *                       beside the resident fields even with nothing else in
 *                       flight (it is failed at the head of the queue instead
 *                       of blocking it).  A ticket is
 *                       consumed by the successful or failed wait that
 *                       returns its result.
 *   egs_serve_stats     p50 / p99 / mean latency, throughput, counters.
 *   egs_serve_destroy   drains in-flight work and frees everything.
 */
typedef struct egs_server egs_server;
typedef struct {
    size_t hbm_budget_bytes;
    int32_t max_inflight;
    int32_t tile;
    int32_t band;
    int32_t fallback_fp64; /* nonzero: a mixed-precision request whose
                              evaluation returns EGS_ERR_NOT_PD or
                              EGS_ERR_INACCURATE is run again in EGS_FP64
                              (ahead of the queue) and answered from that run;
                              its latency covers both */
    int32_t xband;         /* EGS_MIX_FP32 requests: egs_opts.xband (0 = band) */
} egs_serve_config;
typedef struct {
    double p50_ms, p99_ms, mean_ms, evals_per_s;
    int64_t completed, failed, rejected, inflight_peak, queued;
    size_t bytes_in_use;  /* fields + workspaces in flight now */
    size_t bytes_peak;    /* maximum of bytes_in_use so far (<= the budget) */
    int64_t fallbacks;    /* mixed requests re-run in FP64 (fallback_fp64) */
} egs_serve_stats_t;
egs_status egs_serve_create(const egs_serve_config *cfg, egs_server **out);
egs_status egs_serve_add_field(egs_server *server, const double *locs, const double *z, int64_t n, int64_t *field_id);
egs_status egs_serve_submit(egs_server *server, int64_t field_id, const double theta[3], egs_precision p,
                            int64_t *ticket);
egs_status egs_serve_wait(egs_server *server, int64_t ticket, int32_t timeout_ms, double *out_loglik, egs_info *info);
egs_status egs_serve_stats(egs_server *server, egs_serve_stats_t *stats);
egs_status egs_serve_destroy(egs_server *server);

/*
 * egs_tc_gemm_test - the tensor-core pipeline of the trailing update on its
 * own: C = A B^T with tcgen05.mma (FP32 accumulation in TMEM), operands
 * streamed by TMA.  Exposed so that the MMA/descriptor path can be checked in
 * isolation; the factorisation calls the same kernel template.
 *   A  device, M x K row-major, FP32 (EGS_MIX_TF32: read as TF32) or BF16
 *   B  device, N x K row-major, same type
 *   C  device, M x N row-major FP32, written
 * M % 128 == 0, N % 256 == 0, K % 64 == 0.  Synchronises stream.
 * EGS_ERR_TIMEOUT if a pipeline wait expired (the kernel unwinds cleanly).
 */
egs_status egs_tc_gemm_test(const void *A, const void *B, int32_t M, int32_t N, int32_t K, egs_precision p, float *C,
                            void *stream);

/*
 * egs_tc_gemm_test_withhold - failure detection of the tensor-core pipeline:
 * egs_tc_gemm_test with the TMA loads of one ring stage (withhold_stage >= 0,
 * counted over the whole launch of one CTA) never issued.  The MMA warp's
 * wait for that stage runs out after its bound (2 s), the kernel unwinds
 * (in-flight loads land, TMEM is freed) and the call returns EGS_ERR_TIMEOUT
 * with the context still usable; C is undefined.  The paper has no
 * counterpart: this is a test of the bounded waits every tcgen05 kernel of
 * the library uses.  EGS_ERR_ARG if withhold_stage < 0.
 */
egs_status egs_tc_gemm_test_withhold(const void *A, const void *B, int32_t M, int32_t N, int32_t K, egs_precision p,
                                     float *C, int64_t withhold_stage, void *stream);

/*
 * egs_ozaki_gemm_test - the FP64-accurate product of the EGS_MIX_FP32 band
 * updates on its own: C = A B^T with every row of A and B cut into five exact
 * BF16 slices (row scale a power of two) and the 15 slice products of levels
 * 2..6 accumulated in FP32 on tcgen05 (levels 2 and 3 exactly), combined in
 * FP64.  Error about K 2^-35 max|A_i.| max|B_j.| per entry; exact when every
 * entry of A and B is an integer in [-127, 127].
 *   A  device, M x K row-major FP64;  B  device, N x K row-major FP64
 *   C  device, M x N row-major FP64, written
 * M % 128 == 0, N % 32 == 0, K % 64 == 0, K <= 512.  Synchronises stream;
 * allocates its slices with cudaMallocAsync on stream.
 */
egs_status egs_ozaki_gemm_test(const double *A, const double *B, int32_t M, int32_t N, int32_t K, double *C,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EGS_H */
