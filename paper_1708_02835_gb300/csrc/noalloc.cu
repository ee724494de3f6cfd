// egs_trsv_tiles_noalloc: the forward solve with log-determinant and dot
// product of egs_trsv_tiles, for callers that cannot allocate device memory
// during the call -- for example a host application whose memory manager
// has already reserved the whole device, or a latency-sensitive loop that
// cannot afford the device-wide synchronisation cudaFree implies.  Its
// scratch (the padded solution vector, the per-tile partial sums and the
// status word) lives in one file-scope device array of fixed size instead
// of being allocated per call; the caller still provides the factor, z and y.
#include <mutex>

#include "egs_internal.cuh"

namespace {

constexpr int64_t kMaxPad = 131072;  // T * tile doubles of padded vector
constexpr int64_t kMaxTiles = 2048;  // T, for the 2T partial sums
constexpr size_t kPadBytes = (size_t)kMaxPad * sizeof(double);
constexpr size_t kPartBytes = (size_t)2 * kMaxTiles * sizeof(double);
constexpr size_t kScratchBytes = kPadBytes + kPartBytes + 256;  // + status word

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
// Device address of g_scratch per device ordinal, with the id of the CUDA
// context it was looked up in: cudaDeviceReset (or any destruction of the
// primary context) reloads the module at a new address, and a new context
// id makes the next call look the address up again.
struct ScratchAddr {
    unsigned long long ctx_id;
    void *addr;
};
ScratchAddr g_addr[256] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current CUDA context (0 if unknown).
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)p;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_scratch on the current device, looked up once per
// device and context (with that device current; the pointer checks before
// this call have already made the device's primary context current, and an
// unknown context id only means a fresh lookup).  In host code the symbol
// itself is only a host-side handle, so kernels must be given this address.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev].addr || ctx == 0 || g_addr[dev].ctx_id != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = ScratchAddr{ctx, p};
    }
    *out = g_addr[dev].addr;
    return cudaSuccess;
}

}  // namespace

using namespace egs;

extern "C" egs_status egs_trsv_tiles_noalloc(const void *tiles, int64_t n, int32_t tile, const double *z, double *y,
                                             double *logdet, double *quad, void *stream)
{
    clear_error();
    if (n < 1) return set_error(EGS_ERR_ARG, "n = %lld must be >= 1", (long long)n);
    if (tile < 64 || tile > 1024 || tile % 64) return set_error(EGS_ERR_ARG, "tile = %d must be a multiple of 64 in [64, 1024]", tile);
    if (!tiles || !z || !y) return set_error(EGS_ERR_ARG, "NULL pointer");
    if (!is_device_ptr(tiles) || !is_device_ptr(z) || !is_device_ptr(y))
        return set_error(EGS_ERR_ARG, "egs_trsv_tiles_noalloc: tiles, z and y must be device memory");
    TileGeom g{n, tile, (int)((n + tile - 1) / tile)};
    const int64_t npad = (int64_t)g.T * g.b;
    if (npad > kMaxPad || g.T > kMaxTiles)
        return set_error(EGS_ERR_ARG,
                         "egs_trsv_tiles_noalloc: n = %lld with tile %d pads to %lld entries; the fixed scratch holds "
                         "at most %lld (use egs_trsv_tiles for larger problems)",
                         (long long)n, tile, (long long)npad, (long long)kMaxPad);
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_error(e, "egs_trsv_tiles_noalloc: scratch address");
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)base;
    double *zpad = (double *)ws;
    double *partials = (double *)(ws + kPadBytes);
    DevStatus *st = (DevStatus *)(ws + kPadBytes + kPartBytes);
    // the status word must start as "no failure"; zpad and partials are
    // fully overwritten by the kernels below
    e = cudaMemsetAsync(st, 0xFF, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st->timeout, 0, sizeof(DevStatus) - sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_pad_vector(z, n, zpad, npad, s);
    if (e == cudaSuccess) e = launch_trsv_tiles_f64((const double *)tiles, g, zpad, partials, st, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, zpad, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    DevStatus h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "egs_trsv_tiles_noalloc");
    if (logdet) *logdet = h.result[1];
    if (quad) *quad = h.result[2];
    return EGS_OK;
}
