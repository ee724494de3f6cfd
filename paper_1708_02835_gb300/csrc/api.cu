// C ABI of libegs (declared in include/egs.h): argument checking, workspace
// layout, host<->device staging and the order of the kernel launches that
// make up one evaluation of Eq. 1 by Algorithm 2.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "egs_internal.cuh"

namespace egs {

static thread_local char g_err[512];

void clear_error() { g_err[0] = 0; }

egs_status set_error(egs_status code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

egs_status cuda_error(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return set_error(EGS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(EGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static std::mutex g_alloc_mu;
static Allocator g_alloc{nullptr, nullptr, nullptr};

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

cudaError_t dev_alloc(const Allocator &A, void **p, size_t bytes, cudaStream_t s)
{
    if (!A.alloc) return cudaMallocAsync(p, bytes, s);
    *p = A.alloc(bytes, (void *)s, A.ctx);
    if (!*p) return cudaErrorMemoryAllocation;
    if (((uintptr_t)*p & 255) != 0) {  // the layouts need 256-byte alignment
        A.free(*p, bytes, (void *)s, A.ctx);
        *p = nullptr;
        return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
}

void dev_free(const Allocator &A, void *p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    if (!A.alloc) cudaFreeAsync(p, s);
    else A.free(p, bytes, (void *)s, A.ctx);
}

static bool tile_ok(int32_t b) { return b >= 64 && b <= 1024 && (b % 64) == 0; }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static egs_status check_theta(const double *theta)
{
    if (!theta) return set_error(EGS_ERR_ARG, "theta is NULL");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(theta[i]) || !(theta[i] > 0.0))
            return set_error(EGS_ERR_ARG, "theta[%d] = %g must be finite and > 0", i, theta[i]);
    return EGS_OK;
}


static Layout make_layout(const TileGeom &g)
{
    Layout L;
    size_t off = 0;
    L.tiles = off;
    off += align256(g.ntiles() * g.tile_elems() * sizeof(double));
    L.locs = off;
    off += align256((size_t)2 * g.n * sizeof(double));
    L.z = off;
    off += align256((size_t)g.n * sizeof(double));
    L.zpad = off;
    off += align256((size_t)g.T * g.b * sizeof(double));
    L.partials = off;
    off += align256((size_t)2 * g.T * sizeof(double));
    L.status = off;
    off += align256(sizeof(DevStatus));
    L.mtab = off;
    off += align256(EGS_MT_DOUBLES * sizeof(double));
    L.pctr = off;
    off += align256((size_t)g.T * potrf_diag_scratch_words(g.b) * sizeof(unsigned));
    L.total = off;
    return L;
}


static int mix_fmt(egs_precision p) { return p == EGS_MIX_FP32 ? 3 : (p == EGS_MIX_TF32 ? 2 : 1); }

static MixedLayout make_mixed_layout(const TileGeom &g, int band, egs_precision p)
{
    MixedLayout L;
    const size_t bb = g.tile_elems();
    const size_t npad = (size_t)g.T * g.b;
    size_t off = 0;
    L.f64 = off;
    off += align256(Tiles::f64_tiles(g.T, band) * bb * sizeof(double));
    L.f32 = off;
    off += align256(Tiles::f32_tiles(g.T, band) * bb * sizeof(float));
    L.slots = off;
    off += align256(symv_slots_bytes(g.b, g.T));
    L.panel = off;
    off += 2 * align256(panel_buffer_bytes(g.b, g.T, mix_fmt(p)));
    L.oz = off;
    if (mix_fmt(p) == 3)
        off += 2 * (align256(ozaki_slices_bytes(g.b, g.T)) +
                    align256((size_t)(g.T > 1 ? g.T - 1 : 1) * g.b * sizeof(double)));
    L.l32 = off;  // TF32 / BF16: L_kk in FP32; FP32 mode: L_kk^T in FP64
    off += align256(bb * sizeof(double));
    L.wsp = off;
    if (mix_fmt(p) == 3) off += 2 * align256(2 * bb * sizeof(float));
    L.vinv = off;
    off += align256((size_t)g.T * bb * sizeof(double));
    L.locs = off;
    off += align256((size_t)2 * g.n * sizeof(double));
    L.z = off;
    off += align256((size_t)g.n * sizeof(double));
    L.vec = off;
    off += 7 * align256(npad * sizeof(double));
    L.partials = off;
    off += align256((size_t)2 * g.T * sizeof(double));
    L.status = off;
    off += align256(sizeof(DevStatus));
    L.err = off;
    off += 256;
    L.mtab = off;
    off += align256(EGS_MT_SCRATCH_DOUBLES * sizeof(double));
    L.pctr = off;
    off += align256((size_t)g.T * potrf_diag_scratch_words(g.b) * sizeof(unsigned));
    L.rs = off;
    off += 2 * align256((size_t)(g.T > 1 ? g.T - 1 : 1) * g.b * sizeof(float));
    L.total = off;
    return L;
}

static bool mixed_p(egs_precision p) { return p == EGS_MIX_FP32 || p == EGS_MIX_TF32 || p == EGS_MIX_BF16; }

static void status_init(DevStatus *st, cudaStream_t s)
{
    cudaMemsetAsync(st, 0xFF, sizeof(unsigned long long), s);
    cudaMemsetAsync(&st->timeout, 0, sizeof(DevStatus) - sizeof(unsigned long long), s);
}

int32_t default_tile(int64_t n, egs_precision p)
{
    if (mixed_p(p)) return n <= 16384 ? 256 : 512;
    if (n <= 4096) return 128;
    if (n <= 16384) return 256;
    return 512;
}

egs_status eval_setup(int64_t n, const double *theta, egs_precision p, const egs_opts *opts, EvalSetup *es)
{
    if (n < 1) return set_error(EGS_ERR_ARG, "n = %lld must be >= 1", (long long)n);
    egs_status sc = check_theta(theta);
    if (sc != EGS_OK) return sc;
    if (p != EGS_FP64 && !mixed_p(p)) return set_error(EGS_ERR_UNIMPLEMENTED, "precision %d not built", (int)p);
    int32_t tile = (opts && opts->tile) ? opts->tile : default_tile(n, p);
    if (!tile_ok(tile)) return set_error(EGS_ERR_ARG, "tile = %d must be a multiple of 64 in [64, 1024]", tile);
    es->band = (opts && opts->band > 0) ? opts->band : 2;
    es->xband = (opts && opts->xband > 0) ? opts->xband : es->band;
    if (es->xband < es->band)
        return set_error(EGS_ERR_ARG, "xband = %d must be >= band = %d (or 0)", es->xband, es->band);
    es->refine = (opts && opts->refine) ? (opts->refine < 0 ? 0 : opts->refine) : 1;
    if (mixed_p(p) && tile % 256 != 0)
        return set_error(EGS_ERR_ARG, "mixed precision needs tile %% 256 == 0 (got %d)", tile);
    es->p = p;
    es->g = TileGeom{n, tile, (int)((n + tile - 1) / tile)};
    es->mixed = mixed_p(p) && es->g.T > es->band;
    es->L = make_layout(es->g);
    es->ML = make_mixed_layout(es->g, es->band, p);
    es->need = es->mixed ? es->ML.total : es->L.total;
    es->locs_off = es->mixed ? es->ML.locs : es->L.locs;
    es->z_off = es->mixed ? es->ML.z : es->L.z;
    egs_matern_params_init(theta, &es->P);
    const int dist = opts ? opts->distance : 0;
    if (dist != EGS_DIST_EUCLIDEAN && dist != EGS_DIST_GREAT_CIRCLE)
        return set_error(EGS_ERR_ARG, "distance = %d must be 0 (Euclidean) or 1 (great circle)", dist);
    es->P.metric = dist;
    es->P.radius = EGS_EARTH_RADIUS_KM;
    return EGS_OK;
}

DevStatus *eval_status(const EvalSetup &es, char *ws) { return (DevStatus *)(ws + (es.mixed ? es.ML.status : es.L.status)); }

double *eval_solution(const EvalSetup &es, char *ws)
{
    if (!es.mixed) return (double *)(ws + es.L.zpad);
    const size_t npad = (size_t)es.g.T * es.g.b;
    const size_t stride = align256(npad * sizeof(double)) / sizeof(double);
    return (double *)(ws + es.ML.vec) + 2 * stride;  // mb.x
}

cudaError_t finish_solution(const EvalSetup &es, char *ws, cudaStream_t s)
{
    if (es.mixed) return cudaSuccess;
    const Tiles tl{(double *)(ws + es.L.tiles), nullptr, es.g.b, es.g.T, es.g.T};
    return backward_solve(tl, eval_solution(es, ws), eval_status(es, ws), s, nullptr);
}

cudaError_t eval_enqueue(const EvalSetup &es, const double *dlocs, const double *dz, char *ws, cudaStream_t s,
                         KernelTimer *kt, cudaEvent_t *ev)
{
    const TileGeom &g = es.g;
    const int64_t n = g.n;
    DevStatus *st = eval_status(es, ws);
    status_init(st, s);
    if (es.mixed) {
        const size_t npad = (size_t)g.T * g.b;
        MixedBuffers mb;
        const MixedLayout &ML = es.ML;
        mb.tl = Tiles{(double *)(ws + ML.f64), (float *)(ws + ML.f32), g.b, g.T, es.band};
        mb.slots = (double *)(ws + ML.slots);
        mb.panel[0] = ws + ML.panel;
        mb.panel[1] = ws + ML.panel + align256(panel_buffer_bytes(g.b, g.T, mix_fmt(es.p)));
        double *v = (double *)(ws + ML.vec);
        const size_t stride = align256(npad * sizeof(double)) / sizeof(double);
        mb.zp = v;
        mb.y = v + stride;
        mb.x = v + 2 * stride;
        mb.d = v + 3 * stride;
        mb.res = v + 4 * stride;
        mb.rows = v + 5 * stride;
        mb.cols = v + 6 * stride;
        mb.partials = (double *)(ws + ML.partials);
        mb.err = (int *)(ws + ML.err);
        mb.mtab = (double *)(ws + ML.mtab);
        mb.pctr = (unsigned *)(ws + ML.pctr);
        mb.xband = es.xband;
        for (int i = 0; i < 2; ++i)
            mb.rs[i] = (float *)(ws + ML.rs + i * align256((size_t)(g.T > 1 ? g.T - 1 : 1) * g.b * sizeof(float)));
        mb.l32 = (float *)(ws + ML.l32);
        mb.lt = (double *)(ws + ML.l32);
        mb.wsp = (float *)(ws + ML.wsp);
        mb.vinv = (double *)(ws + ML.vinv);
        const size_t ozb = align256(ozaki_slices_bytes(g.b, g.T));
        const size_t ozh = ozb + align256((size_t)(g.T > 1 ? g.T - 1 : 1) * g.b * sizeof(double));
        for (int i = 0; i < 2; ++i) {
            mb.oz[i] = ws + ML.oz + i * ozh;
            mb.ozs[i] = (double *)(ws + ML.oz + i * ozh + ozb);
        }
        cudaMemsetAsync(mb.err, 0, sizeof(int), s);
        return run_loglik_mixed(dlocs, dlocs + n, dz, n, es.P, mix_fmt(es.p), es.refine, mb, st, s, kt, ev);
    }
    double *tiles = (double *)(ws + es.L.tiles);
    double *zpad = (double *)(ws + es.L.zpad);
    double *partials = (double *)(ws + es.L.partials);
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e = launch_matern_tiles_f64(dlocs, dlocs + n, g, es.P, tiles, s, kt, (double *)(ws + es.L.mtab));
    if (e == cudaSuccess) {
        if (ev) cudaEventRecord(ev[1], s);
        e = launch_potrf_tiles_f64(tiles, g, st, s, kt, (unsigned *)(ws + es.L.pctr));
    }
    if (e == cudaSuccess) {
        if (ev) cudaEventRecord(ev[2], s);
        e = launch_pad_vector(dz, n, zpad, (int64_t)g.T * g.b, s, kt);
    }
    if (e == cudaSuccess) e = launch_trsv_tiles_f64(tiles, g, zpad, partials, st, s, kt);
    if (e == cudaSuccess && ev) cudaEventRecord(ev[3], s);
    return e;
}

bool mixed_result_ok(const EvalSetup &es, const DevStatus &h)
{
    if (!es.mixed || es.refine < 1) return true;
    const double q = h.result[2], q0 = h.result[3];
    const double tol = es.p == EGS_MIX_FP32 ? kRefineTolFp32 : kRefineTol;
    return std::fabs(q - q0) <= tol * std::fabs(q);
}

void fill_info(const EvalSetup &es, const DevStatus &h, egs_info *info)
{
    const int64_t fi = (h.fail_index == kNoFail) ? -1 : (int64_t)h.fail_index;
    std::memset(info, 0, sizeof(*info));
    info->loglik = h.result[0];
    info->logdet = h.result[1];
    info->quad = h.result[2];
    info->fail_index = fi;
    info->fail_tile = fi >= 0 ? fi / es.g.b : -1;
    info->tile = es.g.b;
    info->band = es.mixed ? es.band : es.g.T;
    info->refine_steps = es.mixed ? es.refine : 0;
    info->quad_unrefined = es.mixed ? h.result[3] : h.result[2];
}


static thread_local std::vector<egs_trace_rec> g_trace;

void store_trace(const KernelTimer &kt, cudaEvent_t origin)
{
    g_trace.clear();
    g_trace.reserve(kt.recs.size());
    for (const KernelTimer::Rec &r : kt.recs) {
        float t0 = 0.f, t1 = 0.f;
        if (!r.e || cudaEventElapsedTime(&t0, origin, r.b) != cudaSuccess ||
            cudaEventElapsedTime(&t1, origin, r.e) != cudaSuccess)
            continue;
        g_trace.push_back(egs_trace_rec{r.cls, r.step, r.side, 0, (double)t0, (double)t1});
    }
}

}  // namespace egs


using namespace egs;

extern "C" {

const char *egs_last_error(void) { return g_err; }

egs_status egs_set_allocator(egs_alloc_fn alloc, egs_free_fn free_fn, void *ctx)
{
    g_err[0] = 0;
    if ((alloc == nullptr) != (free_fn == nullptr))
        return set_error(EGS_ERR_ARG, "egs_set_allocator: give both hooks, or neither to restore cudaMallocAsync");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = Allocator{alloc, free_fn, alloc ? ctx : nullptr};
    return EGS_OK;
}

egs_status egs_trace_last(egs_trace_rec *out, int64_t cap, int64_t *count)
{
    if (!count) return set_error(EGS_ERR_ARG, "egs_trace_last: count is NULL");
    if (cap < 0 || (cap > 0 && !out)) return set_error(EGS_ERR_ARG, "egs_trace_last: bad buffer");
    *count = (int64_t)g_trace.size();
    const int64_t m = cap < *count ? cap : *count;
    for (int64_t i = 0; i < m; ++i) out[i] = g_trace[(size_t)i];
    return EGS_OK;
}

const char *egs_version(void) { return "egs 0.1 (sm_103a)"; }

int32_t egs_default_tile(int64_t n, egs_precision p) { return default_tile(n, p); }

size_t egs_tiles_bytes(int64_t n, int32_t tile, egs_precision p, int32_t band)
{
    if (n < 1 || !tile_ok(tile) || (p != EGS_FP64 && !mixed_p(p))) return 0;
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    if (band <= 0) band = 2;
    if (p == EGS_FP64 || g.T <= band) return g.ntiles() * g.tile_elems() * sizeof(double);
    return Tiles::f64_tiles(g.T, band) * g.tile_elems() * sizeof(double) +
           Tiles::f32_tiles(g.T, band) * g.tile_elems() * sizeof(float);
}

size_t egs_loglik_workspace_bytes(int64_t n, int32_t tile, egs_precision p, int32_t band)
{
    if (tile == 0) tile = default_tile(n, p);
    if (band <= 0) band = 2;
    if (n < 1 || !tile_ok(tile)) return 0;
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    if (p == EGS_FP64 || (mixed_p(p) && g.T <= band)) return make_layout(g).total;
    if (mixed_p(p) && tile % 256 == 0) return make_mixed_layout(g, band, p).total;
    return 0;
}

egs_status egs_matern_tiles(const double *locs, int64_t n, const double theta[3], int32_t tile,
                            egs_precision p, int32_t band, void *tiles, void *stream)
{
    g_err[0] = 0;
    if (n < 1) return set_error(EGS_ERR_ARG, "n = %lld must be >= 1", (long long)n);
    if (!tile_ok(tile)) return set_error(EGS_ERR_ARG, "tile = %d must be a multiple of 64 in [64, 1024]", tile);
    if (p != EGS_FP64 && !mixed_p(p)) return set_error(EGS_ERR_UNIMPLEMENTED, "precision %d not built", (int)p);
    if (!locs || !tiles) return set_error(EGS_ERR_ARG, "NULL pointer");
    egs_status st = check_theta(theta);
    if (st != EGS_OK) return st;
    if (!is_device_ptr(locs) || !is_device_ptr(tiles))
        return set_error(EGS_ERR_ARG, "egs_matern_tiles: locs and tiles must be device memory");
    egs_matern_params P;
    egs_matern_params_init(theta, &P);
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    if (band <= 0) band = 2;
    cudaStream_t s = (cudaStream_t)stream;
    double *tab = nullptr;  // the general-nu local polynomials (stream-ordered scratch)
    cudaError_t e = cudaSuccess;
    const Allocator A = current_allocator();
    const size_t tab_bytes = EGS_MT_SCRATCH_DOUBLES * sizeof(double);
    if (P.kind == EGS_MATERN_GENERAL) e = dev_alloc(A, (void **)&tab, tab_bytes, s);
    if (e != cudaSuccess) return cuda_error(e, "egs_matern_tiles scratch");
    if (p == EGS_FP64 || g.T <= band) {
        e = launch_matern_tiles_f64(locs, locs + n, g, P, (double *)tiles, s, nullptr, tab);
    } else {
        // band tiles as doubles, then the off-band tiles as floats right after them
        double *f64 = (double *)tiles;
        float *f32 = (float *)(f64 + Tiles::f64_tiles(g.T, band) * g.tile_elems());
        const Tiles tl{f64, f32, g.b, g.T, band};
        e = launch_matern_tiles(locs, locs + n, n, tl, P, s, nullptr, tab);
    }
    dev_free(A, tab, tab_bytes, s);
    if (e != cudaSuccess) return cuda_error(e, "egs_matern_tiles launch");
    return EGS_OK;
}

egs_status egs_potrf_tiles(void *tiles, int64_t n, int32_t tile, int64_t *fail_index, void *stream)
{
    g_err[0] = 0;
    if (n < 1) return set_error(EGS_ERR_ARG, "n = %lld must be >= 1", (long long)n);
    if (!tile_ok(tile)) return set_error(EGS_ERR_ARG, "tile = %d must be a multiple of 64 in [64, 1024]", tile);
    if (!tiles) return set_error(EGS_ERR_ARG, "NULL pointer");
    if (!is_device_ptr(tiles)) return set_error(EGS_ERR_ARG, "egs_potrf_tiles: tiles must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    DevStatus *st = nullptr;
    const size_t sbytes = align256(sizeof(DevStatus));
    const Allocator A = current_allocator();
    const size_t wbytes = sbytes + (size_t)g.T * potrf_diag_scratch_words(g.b) * sizeof(unsigned);
    cudaError_t e = dev_alloc(A, (void **)&st, wbytes, s);
    if (e != cudaSuccess) return cuda_error(e, "egs_potrf_tiles workspace");
    status_init(st, s);
    e = launch_potrf_tiles_f64((double *)tiles, g, st, s, nullptr, (unsigned *)((char *)st + sbytes));
    DevStatus h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
    dev_free(A, st, wbytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "egs_potrf_tiles");
    if (h.timeout) return set_error(EGS_ERR_TIMEOUT, "egs_potrf_tiles: a dependency wait of the diagonal POTRF timed out");
    const int64_t fi = (h.fail_index == kNoFail) ? -1 : (int64_t)h.fail_index;
    if (fail_index) *fail_index = fi;
    if (fi >= 0) return set_error(EGS_ERR_NOT_PD, "not positive definite at row %lld", (long long)fi);
    return EGS_OK;
}

egs_status egs_trsv_tiles(const void *tiles, int64_t n, int32_t tile, const double *z, double *y,
                          double *logdet, double *quad, void *stream)
{
    g_err[0] = 0;
    if (n < 1) return set_error(EGS_ERR_ARG, "n = %lld must be >= 1", (long long)n);
    if (!tile_ok(tile)) return set_error(EGS_ERR_ARG, "tile = %d must be a multiple of 64 in [64, 1024]", tile);
    if (!tiles || !z || !y) return set_error(EGS_ERR_ARG, "NULL pointer");
    if (!is_device_ptr(tiles) || !is_device_ptr(z) || !is_device_ptr(y))
        return set_error(EGS_ERR_ARG, "egs_trsv_tiles: tiles, z and y must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    const size_t npad = (size_t)g.T * g.b;
    char *ws = nullptr;
    const size_t bytes = align256(npad * sizeof(double)) + align256(2 * g.T * sizeof(double)) + align256(sizeof(DevStatus));
    const Allocator A = current_allocator();
    cudaError_t e = dev_alloc(A, (void **)&ws, bytes, s);
    if (e != cudaSuccess) return cuda_error(e, "egs_trsv_tiles workspace");
    double *zpad = (double *)ws;
    double *partials = (double *)(ws + align256(npad * sizeof(double)));
    DevStatus *st = (DevStatus *)(ws + align256(npad * sizeof(double)) + align256(2 * g.T * sizeof(double)));
    status_init(st, s);
    e = launch_pad_vector(z, n, zpad, (int64_t)npad, s);
    if (e == cudaSuccess) e = launch_trsv_tiles_f64((const double *)tiles, g, zpad, partials, st, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, zpad, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    DevStatus h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
    dev_free(A, ws, bytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "egs_trsv_tiles");
    if (logdet) *logdet = h.result[1];
    if (quad) *quad = h.result[2];
    return EGS_OK;
}

egs_status egs_loglik_ex(const double *locs, const double *z, const double theta[3], int64_t n,
                         egs_precision p, const egs_opts *opts, double *out_loglik, egs_info *info,
                         void *stream)
{
    g_err[0] = 0;
    if (out_loglik) *out_loglik = NAN;
    if (!locs || !z) return set_error(EGS_ERR_ARG, "NULL pointer");
    EvalSetup es;
    egs_status sc = eval_setup(n, theta, p, opts, &es);
    if (sc != EGS_OK) return sc;
    const bool timing = opts && opts->timing;
    KernelTimer kt;
    kt.on = opts && opts->timing >= 2;
    cudaStream_t s = (cudaStream_t)stream;
    kt.main = s;

    char *ws = nullptr;
    bool own = false;
    cudaError_t e = cudaSuccess;
    const Allocator A = current_allocator();
    if (opts && opts->workspace) {
        if (opts->workspace_bytes < es.need)
            return set_error(EGS_ERR_ARG, "workspace of %zu bytes < %zu needed", opts->workspace_bytes, es.need);
        ws = (char *)opts->workspace;
    } else {
        e = dev_alloc(A, (void **)&ws, es.need, s);
        if (e != cudaSuccess) return cuda_error(e, "egs_loglik workspace");
        own = true;
    }
    const double *dlocs = locs, *dz = z;
    if (!is_device_ptr(locs)) {
        dlocs = (const double *)(ws + es.locs_off);
        e = cudaMemcpyAsync((void *)dlocs, locs, (size_t)2 * n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess && !is_device_ptr(z)) {
        dz = (const double *)(ws + es.z_off);
        e = cudaMemcpyAsync((void *)dz, z, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timing)
        for (int i = 0; i < 4; ++i) cudaEventCreate(&ev[i]);
    if (e == cudaSuccess) e = eval_enqueue(es, dlocs, dz, ws, s, &kt, timing ? ev : nullptr);
    DevStatus h;
    int herr = 0;
    if (e == cudaSuccess && es.mixed) e = cudaMemcpyAsync(&herr, ws + es.ML.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, eval_status(es, ws), sizeof(h), cudaMemcpyDeviceToHost, s);
    if (own) dev_free(A, ws, es.need, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms[3] = {0, 0, 0};
    if (timing) {
        if (e == cudaSuccess)
            for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        if (e == cudaSuccess && opts->timing >= 3) store_trace(kt, ev[0]);
        for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    }
    if (e != cudaSuccess) return cuda_error(e, "egs_loglik");
    if (herr || h.timeout) return set_error(EGS_ERR_TIMEOUT, "egs_loglik: a bounded device wait timed out");
    if (info) {
        fill_info(es, h, info);
        info->launches = kt.launches;
        info->ms_generate = ms[0];
        info->ms_factor = ms[1];
        info->ms_solve = ms[2];
        info->ms_total = (double)ms[0] + ms[1] + ms[2];
        info->ms_potrf = kt.ms(KC_POTRF);
        info->ms_trsm = kt.ms(KC_TRSM);
        info->ms_update = kt.ms(KC_UPDATE);
        info->ms_trsv = kt.ms(KC_TRSV);
        info->ms_update_f64 = kt.ms(KC_UPDATE64);
    }
    const int64_t fi = (h.fail_index == kNoFail) ? -1 : (int64_t)h.fail_index;
    if (fi >= 0) return set_error(EGS_ERR_NOT_PD, "not positive definite at row %lld (tile %lld)", (long long)fi,
                                  (long long)(fi / es.g.b));
    if (!mixed_result_ok(es, h))
        return set_error(EGS_ERR_INACCURATE,
                         "the refinement step changed the quadratic form by %.3g relative (limit %g): the mixed "
                         "factor is too inexact for this Sigma; evaluate in EGS_FP64",
                         std::fabs(h.result[2] - h.result[3]) / std::fabs(h.result[2]),
                         es.p == EGS_MIX_FP32 ? kRefineTolFp32 : kRefineTol);
    if (out_loglik) *out_loglik = h.result[0];
    return EGS_OK;
}

egs_status egs_simulate(const double *locs, const double *e, const double theta[3], int64_t n, int32_t tile, double *z,
                        void *stream)
{
    g_err[0] = 0;
    if (!locs || !e || !z) return set_error(EGS_ERR_ARG, "NULL pointer");
    if (!is_device_ptr(z)) return set_error(EGS_ERR_ARG, "egs_simulate: z must be device memory");
    EvalSetup es;
    egs_opts o{};
    o.tile = tile;
    egs_status sc = eval_setup(n, theta, EGS_FP64, &o, &es);
    if (sc != EGS_OK) return sc;
    cudaStream_t s = (cudaStream_t)stream;
    const TileGeom &g = es.g;
    char *ws = nullptr;
    const Allocator A = current_allocator();
    cudaError_t err = dev_alloc(A, (void **)&ws, es.need, s);
    if (err != cudaSuccess) return cuda_error(err, "egs_simulate workspace");
    double *tiles = (double *)(ws + es.L.tiles);
    double *epad = (double *)(ws + es.L.zpad);
    DevStatus *st = eval_status(es, ws);
    const double *dlocs = locs, *de = e;
    if (!is_device_ptr(locs)) {
        dlocs = (const double *)(ws + es.L.locs);
        err = cudaMemcpyAsync((void *)dlocs, locs, (size_t)2 * n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (err == cudaSuccess && !is_device_ptr(e)) {
        de = (const double *)(ws + es.L.z);
        err = cudaMemcpyAsync((void *)de, e, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    double *zfull = nullptr;
    const size_t zbytes = (size_t)g.T * g.b * sizeof(double);
    if (err == cudaSuccess) err = dev_alloc(A, (void **)&zfull, zbytes, s);
    if (err == cudaSuccess) {
        status_init(st, s);
        err = launch_matern_tiles_f64(dlocs, dlocs + n, g, es.P, tiles, s, nullptr, (double *)(ws + es.L.mtab));
    }
    if (err == cudaSuccess) err = launch_potrf_tiles_f64(tiles, g, st, s, nullptr, (unsigned *)(ws + es.L.pctr));
    if (err == cudaSuccess) err = launch_pad_vector(de, n, epad, (int64_t)g.T * g.b, s);
    if (err == cudaSuccess) err = launch_trmv_lower(tiles, g, epad, zfull, st, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(z, zfull, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    DevStatus h;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
    dev_free(A, zfull, zbytes, s);
    dev_free(A, ws, es.need, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return cuda_error(err, "egs_simulate");
    if (h.timeout) return set_error(EGS_ERR_TIMEOUT, "egs_simulate: a bounded device wait timed out");
    if (h.fail_index != kNoFail)
        return set_error(EGS_ERR_NOT_PD, "egs_simulate: not positive definite at row %lld",
                         (long long)h.fail_index);
    return EGS_OK;
}

egs_status egs_loglik(const double *locs, const double *z, const double theta[3], int64_t n, egs_precision p,
                      double *out_loglik, egs_info *info, void *stream)
{
    return egs_loglik_ex(locs, z, theta, n, p, nullptr, out_loglik, info, stream);
}

}  // extern "C"
