// The FP64 refinement residual of the mixed precisions without a stored copy
// of Sigma: r = Z - Sigma x with every entry of Sigma(theta) (Eq. 2)
// regenerated tile by tile while it is multiplied.  The entries are formed in
// double-float arithmetic (matern_df.cuh, about 1e-14 relative: the same
// values the generator rounds into the FP32 tiles) or, for the great-circle
// distance and theta outside the float range, by the direct FP64 evaluation.
//
// One CTA per lower tile (i, j): it evaluates the tile's b x b entries once
// and uses each twice, for the rows part sum_j Sigma_ij x_j and, below the
// diagonal, for the columns part sum_i Sigma_ij x_i of the symmetric product
// (the diagonal tiles hold both triangles and contribute rows only).  Thread
// (ty, tx) of 16 x 16 owns 4 x 4 entries of each 64 x 64 sub-block; its
// partial sums are combined across threads in shared memory in a fixed
// order, and the tile's b row sums and b column sums are written as FP64 to
// slots (row sums of tile (i, j) at slot j, column sums at slot i), which
// k_residual_slots adds in slot order: every result is deterministic.
#include "egs_internal.cuh"
#include "matern.cuh"
#include "matern_df.cuh"

namespace egs {

namespace {

__device__ __forceinline__ bool sfailed(const DevStatus *st)
{
    return *(volatile const unsigned long long *)&st->fail_index != kNoFail;
}

__device__ __forceinline__ void tile_index(int64_t t, int &i, int &j)
{
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    i = ii;
    j = (int)(t - (int64_t)ii * (ii + 1) / 2);
}

__device__ __forceinline__ df::F2 split_df(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ float4 split_pt(double x, double y)
{
    const float xh = __double2float_rn(x), yh = __double2float_rn(y);
    return make_float4(xh, __double2float_rn(x - (double)xh), yh, __double2float_rn(y - (double)yh));
}

// Shared-memory layout of k_symv_regen (b <= 1024).
struct SymvSmem {
    static constexpr size_t pts(int b) { return (size_t)b * sizeof(float4); }
    static constexpr size_t vec(int b) { return (size_t)b * sizeof(float2); }
    static size_t bytes(int b, bool general)
    {
        return 2 * pts(b) + 4 * vec(b) + 16 * 64 * sizeof(float2) + 2 * EGS_DF_TAB * sizeof(float) +
               (general ? EGS_MT_DOUBLES * sizeof(float2) : 0);
    }
};

// EV: 0 double-float closed forms, 1 double-float local polynomials (general
// nu), 2 direct FP64 evaluation (tabd: the FP64 polynomials of a general nu).
template <int EV>
__global__ void __launch_bounds__(256)
k_symv_regen(const double *__restrict__ X, const double *__restrict__ Y, int64_t n, int b, int64_t npad,
             const __grid_constant__ egs_matern_df Dg, const __grid_constant__ egs_matern_params Pg,
             const float2 *__restrict__ ctab_g, const double *__restrict__ tabd, const double *__restrict__ x,
             double *__restrict__ prow, double *__restrict__ pcol, const DevStatus *st)
{
    if (sfailed(st)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *rp = reinterpret_cast<float4 *>(smem);                 // row locations, split
    float4 *cp = rp + b;                                           // column locations, split
    float2 *xr = reinterpret_cast<float2 *>(cp + b);               // x of the tile's rows
    float2 *xc = xr + b;                                           // x of the tile's columns
    float2 *racc = xc + b;                                         // row sums
    float2 *cacc = racc + b;                                       // column sums
    float2 *red = cacc + b;                                        // 16 x 64 partial sums
    float *etab = reinterpret_cast<float *>(red + 16 * 64);
    float2 *ctab = reinterpret_cast<float2 *>(etab + 2 * EGS_DF_TAB);

    int ti, tj;
    tile_index((int64_t)blockIdx.x, ti, tj);
    const bool diag = ti == tj;
    const int64_t r0 = (int64_t)ti * b, c0 = (int64_t)tj * b;
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const int64_t gi = r0 + i, gj = c0 + i;
        rp[i] = gi < n ? split_pt(X[gi], Y[gi]) : make_float4(0.f, 0.f, 0.f, 0.f);
        cp[i] = gj < n ? split_pt(X[gj], Y[gj]) : make_float4(0.f, 0.f, 0.f, 0.f);
        const df::F2 a = split_df(x[gi]), c = split_df(x[gj]);
        xr[i] = make_float2(a.h, a.l);
        xc[i] = make_float2(c.h, c.l);
        racc[i] = make_float2(0.f, 0.f);
        cacc[i] = make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < 2 * EGS_DF_TAB; i += blockDim.x) etab[i] = Dg.tab[i];
    if (EV == 1)
        for (int i = threadIdx.x; i < EGS_MT_DOUBLES; i += blockDim.x) ctab[i] = ctab_g[i];
    __syncthreads();
    const df::Consts C{{Dg.inv_th2[0], Dg.inv_th2[1]}, Dg.kind};
    const df::F2 th1 = EV == 2 ? split_df(Pg.th1) : df::F2{Dg.tab[0], Dg.tab[1]};  // theta1 (= theta1 2^0)
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int nsub = b >> 6;
    for (int sr = 0; sr < nsub; ++sr) {
        df::F2 ra[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int sc = 0; sc < nsub; ++sc) {
            df::F2 ca[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int r = sr * 64 + ty * 4 + a;
                const int64_t gi = r0 + r;
                const float4 pi = rp[r];
                const df::F2 xi{xr[r].x, xr[r].y};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = sc * 64 + tx * 4 + q;
                    const int64_t gj = c0 + c;
                    df::F2 v;
                    if (gi >= n || gj >= n) {
                        v = {gi == gj ? 1.0f : 0.0f, 0.0f};
                    } else if (gi == gj) {
                        v = th1;
                    } else if (EV == 2) {
                        v = split_df(matern_eval(&Pg, loc_dist(&Pg, X[gi], Y[gi], X[gj], Y[gj]) * Pg.inv_th2, tabd));
                    } else {
                        v = df::matern_entry_df<EV == 1>(C, pi, cp[c], etab, ctab, &Pg);
                    }
                    ra[a] = df::mul_add(v, df::F2{xc[c].x, xc[c].y}, ra[a]);
                    ca[q] = df::mul_add(v, xi, ca[q]);
                }
            }
            if (!diag) {
                // column sums of this sub-block: 16 row groups, added in order
#pragma unroll
                for (int q = 0; q < 4; ++q) red[ty * 64 + tx * 4 + q] = make_float2(ca[q].h, ca[q].l);
                __syncthreads();
                if (threadIdx.x < 64) {
                    df::F2 s{cacc[sc * 64 + threadIdx.x].x, cacc[sc * 64 + threadIdx.x].y};
                    for (int g = 0; g < 16; ++g) s = df::add(s, df::F2{red[g * 64 + threadIdx.x].x, red[g * 64 + threadIdx.x].y});
                    cacc[sc * 64 + threadIdx.x] = make_float2(s.h, s.l);
                }
                __syncthreads();
            }
        }
        // row sums of this block row: 16 column groups, added in order
#pragma unroll
        for (int a = 0; a < 4; ++a) red[tx * 64 + ty * 4 + a] = make_float2(ra[a].h, ra[a].l);
        __syncthreads();
        if (threadIdx.x < 64) {
            df::F2 s{0.f, 0.f};
            for (int g = 0; g < 16; ++g) s = df::add(s, df::F2{red[g * 64 + threadIdx.x].x, red[g * 64 + threadIdx.x].y});
            racc[sr * 64 + threadIdx.x] = make_float2(s.h, s.l);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        prow[(size_t)tj * npad + r0 + i] = (double)racc[i].x + (double)racc[i].y;
        if (!diag) pcol[(size_t)ti * npad + c0 + i] = (double)cacc[i].x + (double)cacc[i].y;
    }
}

// d = z - Sigma x from the slots: row sums of tiles (i, 0 .. i), then the
// column sums of tiles (i + 1 .. T - 1, i), in slot order.
__global__ void k_residual_slots(const double *__restrict__ zp, const double *__restrict__ prow,
                                 const double *__restrict__ pcol, int b, int T, int64_t npad, double *__restrict__ d,
                                 const DevStatus *st)
{
    if (sfailed(st)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    const int t = (int)(i / b);
    double s = 0.0;
    for (int j = 0; j <= t; ++j) s += prow[(size_t)j * npad + i];
    for (int m = t + 1; m < T; ++m) s += pcol[(size_t)m * npad + i];
    d[i] = zp[i] - s;
}

}  // namespace

size_t symv_slots_bytes(int b, int T) { return (size_t)2 * T * (size_t)T * b * sizeof(double); }

cudaError_t launch_residual_regen(const double *X, const double *Y, int64_t n, int b, int T,
                                  const egs_matern_params &P, double *tab, const double *x, const double *zp,
                                  double *slots, double *d, const DevStatus *st, cudaStream_t s, KernelTimer *kt)
{
    const int64_t npad = (int64_t)T * b;
    double *prow = slots, *pcol = slots + (size_t)T * npad;
    egs_matern_df D;
    const bool dfp = matern_df_applies(P, tab != nullptr, &D);
    const int ev = dfp ? (P.kind == EGS_MATERN_GENERAL ? 1 : 0) : 2;
    const size_t sm = SymvSmem::bytes(b, ev == 1);
    const unsigned grid = (unsigned)((size_t)T * (T + 1) / 2);
    const double *tabd = (P.kind == EGS_MATERN_GENERAL) ? tab : nullptr;
    const float2 *ctab = ev == 1 ? matern_df_table(tab) : nullptr;
    cudaError_t e = cudaSuccess;
    if (ev == 0) {
        e = cudaFuncSetAttribute(k_symv_regen<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            EGS_LAUNCH(kt, KC_OTHER, s, k_symv_regen<0><<<grid, 256, sm, s>>>(X, Y, n, b, npad, D, P, ctab, tabd, x,
                                                                               prow, pcol, st));
    } else if (ev == 1) {
        e = cudaFuncSetAttribute(k_symv_regen<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            EGS_LAUNCH(kt, KC_OTHER, s, k_symv_regen<1><<<grid, 256, sm, s>>>(X, Y, n, b, npad, D, P, ctab, tabd, x,
                                                                               prow, pcol, st));
    } else {
        e = cudaFuncSetAttribute(k_symv_regen<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            EGS_LAUNCH(kt, KC_OTHER, s, k_symv_regen<2><<<grid, 256, sm, s>>>(X, Y, n, b, npad, D, P, ctab, tabd, x,
                                                                               prow, pcol, st));
    }
    if (e != cudaSuccess) return e;
    const unsigned vb = (unsigned)((npad + 255) / 256);
    EGS_LAUNCH(kt, KC_OTHER, s, k_residual_slots<<<vb, 256, 0, s>>>(zp, prow, pcol, b, T, npad, d, st));
    return cudaGetLastError();
}

}  // namespace egs
