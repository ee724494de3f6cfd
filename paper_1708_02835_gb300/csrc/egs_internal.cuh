// Internal declarations shared by the CUDA translation units of libegs.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda.h>
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

// Storage of the lower tiles.  Dense FP64 mode (band >= T): every tile is
// double, tile (i, j) at position i (i + 1) / 2 + j of f64.  Mixed mode:
// tiles with i - j < band are double in f64 at position i * band + (i - j);
// the others are float in f32 at position (i - band)(i - band + 1) / 2 + j.
struct Tiles {
    double *f64;
    float *f32;
    int b, T, band;
    __host__ __device__ bool dense() const { return band >= T; }
    __host__ __device__ bool is64(int i, int j) const { return i - j < band; }
    __host__ __device__ size_t bb() const { return (size_t)b * (size_t)b; }
    __host__ __device__ double *t64(int i, int j) const
    {
        return dense() ? f64 + (size_t)tile_linear(i, j) * bb() : f64 + ((size_t)i * band + (i - j)) * bb();
    }
    __host__ __device__ float *t32(int i, int j) const
    {
        const int64_t r = i - band;
        return f32 + ((size_t)(r * (r + 1) / 2) + (size_t)j) * bb();
    }
    static size_t f64_tiles(int T, int band) { return band >= T ? (size_t)T * (T + 1) / 2 : (size_t)T * band; }
    static size_t f32_tiles(int T, int band)
    {
        if (band >= T) return 0;
        const size_t r = (size_t)(T - band);
        return r * (r + 1) / 2;
    }
};

// Geometry of a lower-tile matrix.
struct TileGeom {
    int64_t n;
    int b;
    int T;
    size_t tile_elems() const { return (size_t)b * (size_t)b; }
    size_t ntiles() const { return (size_t)T * (size_t)(T + 1) / 2; }
};

// Kernel classes for per-class device timing.
// KC_UPDATE64: the FP64 update launches of the mixed-precision factorisation.
enum KernelClass { KC_GEN = 0, KC_POTRF, KC_TRSM, KC_UPDATE, KC_TRSV, KC_OTHER, KC_UPDATE64, KC_COUNT };

// Counts launches and, when enabled, brackets each launch with a CUDA event
// pair on the launching stream so the summed duration of each kernel class
// can be read after the stream has finished.
struct KernelTimer {
    bool on = false;
    int launches = 0;
    int step = -1;                // factorisation step of the launches that follow (-1: none)
    cudaStream_t main = nullptr;  // the call's stream; any other counts as the side stream
    struct Rec {
        int cls, step, side;
        cudaEvent_t b, e;
    };
    std::vector<Rec> recs;  // one per launch, in enqueue order
    void begin(int cls, cudaStream_t s)
    {
        if (!on) return;
        Rec r{cls, step, s != main ? 1 : 0, nullptr, nullptr};
        cudaEventCreate(&r.b);
        cudaEventRecord(r.b, s);
        recs.push_back(r);
    }
    void end(int cls, cudaStream_t s)
    {
        (void)cls;
        ++launches;
        if (!on || recs.empty()) return;
        cudaEventCreate(&recs.back().e);
        cudaEventRecord(recs.back().e, s);
    }
    // Summed milliseconds of a class (call after the stream has finished).
    double ms(int cls) const
    {
        double t = 0.0;
        for (const Rec &r : recs) {
            float x = 0.f;
            if (r.cls == cls && r.e && cudaEventElapsedTime(&x, r.b, r.e) == cudaSuccess) t += x;
        }
        return t;
    }
    ~KernelTimer()
    {
        for (const Rec &r : recs) {
            if (r.b) cudaEventDestroy(r.b);
            if (r.e) cudaEventDestroy(r.e);
        }
    }
};

// Per-launch trace of the calling thread's last egs_loglik_ex with
// timing >= 3 (start and end relative to the start of Sigma generation).
void store_trace(const KernelTimer &kt, cudaEvent_t origin);

#define EGS_LAUNCH(kt, cls, s, ...)      \
    do {                                 \
        if (kt) (kt)->begin((cls), (s)); \
        __VA_ARGS__;                     \
        if (kt) (kt)->end((cls), (s));   \
    } while (0)

// Device memory of the library's calls: the caller's hooks (egs_set_allocator)
// or cudaMallocAsync / cudaFreeAsync.  An allocation is freed with the
// Allocator value that made it.
struct Allocator {
    egs_alloc_fn alloc;  // NULL: cudaMallocAsync
    egs_free_fn free;
    void *ctx;
};
Allocator current_allocator();
cudaError_t dev_alloc(const Allocator &A, void **p, size_t bytes, cudaStream_t s);
void dev_free(const Allocator &A, void *p, size_t bytes, cudaStream_t s);

// True for device (or managed) memory; host pointers are staged by the calls.
bool is_device_ptr(const void *p);

// Error reporting (api.cu): thread-local message, returns code.  clear_error
// empties the message at the start of a call.
void clear_error();
egs_status set_error(egs_status code, const char *fmt, ...);
egs_status cuda_error(cudaError_t e, const char *what);

// ---- launchers (stream-ordered, no synchronisation) ----
// Sigma(theta) into FP64 lower tiles.  tab: EGS_MT_DOUBLES doubles of device
// scratch for the local polynomials of a general nu (built first on s), or
// NULL to evaluate every entry directly.
cudaError_t launch_matern_tiles_f64(const double *X, const double *Y, const TileGeom &g,
                                    const egs_matern_params &P, double *tiles, cudaStream_t s,
                                    KernelTimer *kt = nullptr, double *tab = nullptr);
// The local polynomials of a general nu into tab (EGS_MT_DOUBLES doubles).
cudaError_t launch_matern_table(const egs_matern_params &P, double *tab, cudaStream_t s, KernelTimer *kt = nullptr);

// Tile Cholesky in place (FP64).  Stops doing work once st->fail_index is set.
// ctr: T * potrf_diag_scratch_words(b) words of device scratch for the
// one-launch diagonal POTRFs (zeroed here).
cudaError_t launch_potrf_tiles_f64(double *tiles, const TileGeom &g, DevStatus *st, cudaStream_t s,
                                   KernelTimer *kt, unsigned *ctr);
// Counter words one diagonal tile's one-launch POTRF needs.
size_t potrf_diag_scratch_words(int b);

// Forward solve L y = z in place on zpad (T*b doubles, padded with zeros),
// with per-tile log-det / dot partials and the final assembly into st->result.
cudaError_t launch_trsv_tiles_f64(const double *tiles, const TileGeom &g, double *zpad, double *partials,
                                  DevStatus *st, cudaStream_t s, KernelTimer *kt = nullptr);

// Sigma(theta) into any Tiles storage.  For
// a mixed layout with the Euclidean distance the off-band tiles are evaluated
// in double-float arithmetic (matern_df.cuh); tab must then hold
// EGS_MT_SCRATCH_DOUBLES doubles (the general-nu polynomials and their
// float-pair split).
cudaError_t launch_matern_tiles(const double *X, const double *Y, int64_t n, const Tiles &tl,
                                const egs_matern_params &P, cudaStream_t s, KernelTimer *kt, double *tab = nullptr);

// The double-float evaluation applies to these parameters (Euclidean
// distance; a general nu needs the polynomial table); fills D.
bool matern_df_applies(const egs_matern_params &P, bool have_table, egs_matern_df *D);
// The float-pair copy of the general-nu polynomials inside a generator scratch.
float2 *matern_df_table(double *tab);

// Mixed-precision evaluation buffers (all device, sized by mixed_layout).
struct MixedBuffers {
    Tiles tl;
    double *slots;    // 2 T * T b doubles: per-tile row and column sums of the refinement residual
    void *panel[2];   // two operand buffers of panel_buffer_bytes each, step k uses k % 2
    double *zp, *y, *x, *d, *res, *rows, *cols;  // T*b vectors
    double *partials; // 2T
    int *err;
    float *l32;       // b x b: L_kk rounded to FP32 for the off-band TRSM of step k (TF32 / BF16 modes)
    double *lt;       // b x b, the same region: L_kk^T of step k (FP32 mode, for the inversion)
    float *wsp;       // FP32 mode: W = L_kk^-1 in split-TF32 layout, b rows of [hi | lo] (2b); two such
                      // buffers of 2 b^2 floats, step k uses k % 2
    double *vinv;     // T b x b: V_k = L_kk^-T (upper triangular) for the solves
    void *oz[2];      // FP32 mode: BF16 slices of the panel rows (ozaki_slices_bytes), step k uses k % 2
    double *ozs[2];   // FP32 mode: their row scales, (T-1) b doubles each
    double *mtab;     // EGS_MT_SCRATCH_DOUBLES: the generator's local polynomials (general nu)
    unsigned *pctr;   // T * potrf_diag_scratch_words(b): counters of the one-launch diagonal POTRFs
    float *rs[2];     // FP32 mode: the power-of-two scales of the split-FP16 panel rows, (T-1) b each
    int xband;        // FP32 mode: tiles with i - j < xband get FP64-accurate updates (>= tl.band)
};

// The refinement residual d = zp - Sigma x (T b padded vectors) with Sigma(theta)
// regenerated tile by tile (symv_regen.cu): no stored copy of Sigma.  slots:
// symv_slots_bytes(b, T) of device scratch; tab: the generator's scratch of
// this evaluation (general nu: its polynomials, built by the generation).
size_t symv_slots_bytes(int b, int T);
cudaError_t launch_residual_regen(const double *X, const double *Y, int64_t n, int b, int T,
                                  const egs_matern_params &P, double *tab, const double *x, const double *zp,
                                  double *slots, double *d, const DevStatus *st, cudaStream_t s, KernelTimer *kt);

// One mixed-precision evaluation (fmt 3 = split TF32, 2 = TF32, 1 = BF16); the
// result lands in st->result (loglik, logdet, quad refined, quad unrefined).
cudaError_t run_loglik_mixed(const double *X, const double *Y, const double *z, int64_t n, const egs_matern_params &P,
                             int fmt, int refine, const MixedBuffers &mb, DevStatus *st, cudaStream_t s, KernelTimer *kt,
                             cudaEvent_t *phase_ev);

// Layouts and setup of one evaluation (api.cu), shared with the serving loop.
struct Layout {
    size_t tiles, locs, z, zpad, partials, status, mtab, pctr, total;
};
struct MixedLayout {
    size_t f64, f32, slots, panel, oz, l32, wsp, vinv, locs, z, vec, partials, status, err, mtab, pctr, rs, total;
};
struct EvalSetup {
    TileGeom g;
    int band, refine, xband;
    bool mixed;
    egs_precision p;
    Layout L;
    MixedLayout ML;
    size_t need, locs_off, z_off;
    egs_matern_params P;
};
egs_status eval_setup(int64_t n, const double *theta, egs_precision p, const egs_opts *opts, EvalSetup *es);
// Enqueue one evaluation on s; inputs on the device, ws holds es.need bytes.
cudaError_t eval_enqueue(const EvalSetup &es, const double *dlocs, const double *dz, char *ws, cudaStream_t s,
                         KernelTimer *kt, cudaEvent_t *ev);
DevStatus *eval_status(const EvalSetup &es, char *ws);
// After eval_enqueue: mixed -> x = Sigma^-1 Z (refined); FP64 -> y = L^-1 Z
// (finish_solution turns it into Sigma^-1 Z with the backward solve).
double *eval_solution(const EvalSetup &es, char *ws);
cudaError_t finish_solution(const EvalSetup &es, char *ws, cudaStream_t s);
void fill_info(const EvalSetup &es, const DevStatus &h, egs_info *info);
// Mixed precision with refinement: was the FP64 refinement step small?
// |quad - quad_unrefined| <= tol |quad| with tol = kRefineTolFp32 in the FP32
// mode (measured: returned l then within ~2.5 tol of FP64) and kRefineTol in
// TF32 / BF16 (a guard against gross errors only: their log-determinant
// error is not seen by the refinement); always true otherwise.
constexpr double kRefineTol = 1e-3;
constexpr double kRefineTolFp32 = 1e-5;
bool mixed_result_ok(const EvalSetup &es, const DevStatus &h);
int32_t default_tile(int64_t n, egs_precision p);

// Building blocks shared by the FP64 and mixed drivers.
// POTRF of diagonal tile k: one launch over the task graph of its 32 x 32
// blocks; ctr: zeroed potrf_diag_scratch_words(b) words for its counters.
cudaError_t launch_potrf_diag(const Tiles &tl, int k, DevStatus *st, cudaStream_t s, KernelTimer *kt, unsigned *ctr);
cudaError_t launch_trsm_f64(const Tiles &tl, int k, int nrows, DevStatus *st, cudaStream_t s, KernelTimer *kt);
// FP64 update of the first ntri tiles of step k's trailing triangle (row order).
cudaError_t launch_update_f64(const Tiles &tl, int k, int64_t ntri, DevStatus *st, cudaStream_t s, KernelTimer *kt,
                              int cls = KC_UPDATE);
// FP32 mixed mode: FP64-accurate updates of the band tiles whose panel
// operands are not both FP64 band tiles, by exact BF16 slicing on tcgen05
// (ozaki.cu).  The TRSM stage writes the slices of every panel row.
size_t ozaki_slices_bytes(int b, int T);
cudaError_t make_ozaki_maps(const void *oz, int b, int T, CUtensorMap *mapA, CUtensorMap *mapB);
// Band tiles of columns col0 .. col0 + ncols - 1 at step k.
// xband >= tl.band: outputs m = n .. n + xband - 1 (those with m - n >= band
// are FP32 tiles, updated in FP64 and rounded once).
cudaError_t launch_band_out_ozaki(const CUtensorMap &mapA, const CUtensorMap &mapB, const Tiles &tl, int xband, int k,
                                  int col0, int ncols, const double *scale, int *err, cudaStream_t s, KernelTimer *kt);
// The band x band update of step k (tiles (m, n), k < n <= m <= k + nb) from
// the slices of the FP64 band rows.
cudaError_t launch_band_band_ozaki(const CUtensorMap &mapA, const CUtensorMap &mapB, const Tiles &tl, int k, int nb,
                                   const double *scale, int *err, cudaStream_t s, KernelTimer *kt);
cudaError_t launch_forward_solve(const Tiles &tl, double *zpad, double *partials, DevStatus *st, cudaStream_t s,
                                 KernelTimer *kt);
// z_m -= L_mk y_k for m > k, y_k read from ysrc (may equal zpad).
cudaError_t launch_gemv_panel(const Tiles &tl, int k, const double *ysrc, double *zpad, const DevStatus *st,
                              cudaStream_t s, KernelTimer *kt);
// L^T x = v in place (any Tiles storage).
cudaError_t backward_solve(const Tiles &tl, double *v, const DevStatus *st, cudaStream_t s, KernelTimer *kt);
cudaError_t launch_finalize(const double *partials, int T, int64_t n, DevStatus *st, cudaStream_t s, KernelTimer *kt);

// Z = L e over FP64 lower tiles (diagonal tiles with a zero upper triangle).
cudaError_t launch_trmv_lower(const double *tiles, const TileGeom &g, const double *epad, double *out,
                              const DevStatus *st, cudaStream_t s);

// Copy z (n doubles) into zpad (T*b doubles), zero padding.
cudaError_t launch_pad_vector(const double *z, int64_t n, double *zpad, int64_t npad, cudaStream_t s,
                              KernelTimer *kt = nullptr);

// Operand formats of the tensor-core update: 1 = BF16, 2 = TF32 (FP32
// storage), 3 = split TF32 (each panel row holds [hi | lo], hi = tf32(x),
// lo = tf32(x - hi); the update forms lo hi^T + hi lo^T + hi hi^T per K
// slice, an FP32-accurate product), 4 = split FP16 (each row x scaled by the
// power of two s with max |x / s| < 2^15, [hi | lo] = FP16 parts of x / s;
// the same three products at the FP16 rate, times s_m s_n in the epilogue).
// Bytes of one panel buffer ((T-1) * b rows) in format fmt.
size_t panel_buffer_bytes(int b, int T, int fmt);
// Tensor maps over one panel buffer and the tcgen05 trailing update of step k.
cudaError_t make_panel_maps(const void *panel, int fmt, int b, int T, CUtensorMap *mapA, CUtensorMap *mapB);
// Map for the epilogue's TMA reduce into the off-band FP32 tiles.
cudaError_t make_offband_map(const float *f32, int b, size_t ntiles, CUtensorMap *mapC);
// part 0: all trailing tiles of step k; 1: column k + 1; 2: columns k + 2 onwards.
// fmt 3 updates only the off-band outputs (m - n >= band); the band outputs
// are left to the FP64 kernels.
// FP32 mode: the off-band panel TRSM of step k (tiles m0 .. T - 1) on the
// tensor cores, X = A W^T with W = L_kk^-1 (mapW over its split-TF32 B
// layout, make_trsm_w_map) and A in split-TF32 A layout behind mapA; X
// overwrites the FP32 tiles.
cudaError_t make_trsm_w_map(const float *wsp, int b, CUtensorMap *mapW);
cudaError_t launch_trsm_tc(const CUtensorMap &mapA, const CUtensorMap &mapW, const CUtensorMap &mapC, const Tiles &tl,
                           int k, int m0, int *err, cudaStream_t s, KernelTimer *kt);
// fmt 4 (split FP16, the FP32 mode's update): rs holds the power-of-two
// scale of every panel row (panel_f16_scales); NULL otherwise.
// xband (fmt >= 3): outputs with m - n < xband are left to the FP64-accurate kernels.
cudaError_t launch_update_tc(const CUtensorMap &mapA, const CUtensorMap &mapB, const CUtensorMap &mapC, int fmt,
                             const Tiles &tl, int k, int *err, cudaStream_t s, KernelTimer *kt, int part = 0,
                             const float *rs = nullptr, int xband = 0);

}  // namespace egs
