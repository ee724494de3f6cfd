// Matern tile generator (Eq. 2; Algorithm 2, genCovMatrix): writes Sigma(theta)
// directly into the lower-tile layout.  The distance matrix of Algorithm 2
// (genDistanceMatrix) is never stored: each entry's distance is formed in
// registers from the SoA coordinates.
//
// One CTA writes a 64 x 64 sub-block of one tile; a warp writes 32 consecutive
// columns of one row (256 contiguous bytes), so stores are fully coalesced.
#include "egs_internal.cuh"
#include "matern.cuh"
#include "matern_df.cuh"

namespace egs {

// Copy the per-launch constants into shared memory (all later reads are
// warp-uniform broadcasts).
__device__ __forceinline__ void stage_params(const egs_matern_params *src, egs_matern_params *dst)
{
    const double *s = reinterpret_cast<const double *>(src);
    double *d = reinterpret_cast<double *>(dst);
    constexpr int words = (int)(sizeof(egs_matern_params) / sizeof(double));
    for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// Decode lower-tile linear index t -> (i, j), i >= j.
__device__ __forceinline__ void tile_decode(int64_t t, int &i, int &j)
{
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    i = ii;
    j = (int)(t - (int64_t)ii * (ii + 1) / 2);
}

// Writes tile blockIdx.x (lower-tile order) of Sigma into tl: as double when
// the tile is FP64 in tl, else rounded to float.
// tab: the local polynomials of a general nu (built by k_matern_table before
// this launch), staged in shared memory; NULL for the closed forms.
// band_only: blockIdx.x enumerates only the FP64 band tiles of a mixed
// layout, as i * band + (i - j) (slots with j < 0 exit at once).
__global__ void __launch_bounds__(256)
k_matern_tiles(const double *__restrict__ X, const double *__restrict__ Y, int64_t n, Tiles tl,
               const __grid_constant__ egs_matern_params Pg, const double *__restrict__ tab,
               int band_only)
{
    const int b = tl.b;
    __shared__ egs_matern_params Ps;
    __shared__ double Ts[EGS_MT_DOUBLES];
    if (tab)
        for (int i = threadIdx.x; i < EGS_MT_DOUBLES; i += blockDim.x) Ts[i] = tab[i];
    stage_params(&Pg, &Ps);
    const double *T = tab ? Ts : nullptr;
    const egs_matern_params *P = &Ps;
    int ti, tj;
    if (band_only) {
        ti = (int)blockIdx.x / tl.band;
        tj = ti - (int)blockIdx.x % tl.band;
        if (tj < 0) return;
    } else {
        tile_decode((int64_t)blockIdx.x, ti, tj);
    }
    const int nsub = b >> 6;
    const int sr = (int)blockIdx.y / nsub, sc = (int)blockIdx.y % nsub;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int64_t gj = (int64_t)tj * b + sc * 64 + tx;
    double xj = 0.0, yj = 0.0;
    if (gj < n) {
        xj = X[gj];
        yj = Y[gj];
    }
    const double inv_th2 = P->inv_th2;
    const bool is64 = tl.is64(ti, tj);
    double *t64 = is64 ? tl.t64(ti, tj) : nullptr;
    float *t32 = is64 ? nullptr : tl.t32(ti, tj);
    for (int rr = 0; rr < 16; ++rr) {
        const int r = sr * 64 + ty + 4 * rr;
        const int64_t gi = (int64_t)ti * b + r;
        double v;
        if (gi >= n || gj >= n) {
            v = (gi == gj) ? 1.0 : 0.0;
        } else if (gi == gj) {
            v = P->th1;
        } else {
            v = matern_eval(P, loc_dist(P, X[gi], Y[gi], xj, yj) * inv_th2, T);
        }
        const size_t off = (size_t)r * b + sc * 64 + tx;
        if (is64) t64[off] = v;
        else t32[off] = (float)v;
    }
}

// Split a double into a float pair h + l (48 of its 53 bits).
__device__ __forceinline__ float4 split_point(double x, double y)
{
    const float xh = __double2float_rn(x), yh = __double2float_rn(y);
    return make_float4(xh, __double2float_rn(x - (double)xh), yh, __double2float_rn(y - (double)yh));
}

// The off-band (FP32) tiles of a mixed layout in double-float arithmetic
// (matern_df.cuh): the closed forms, or (GENERAL) the local polynomials of a
// general nu, ctab.  grid = (off-band tiles in their storage order, b / 64);
// a CTA covers 64 columns and all b rows of one tile: thread (ty, tx) writes
// column tx of rows ty, ty + 4, ... (coalesced 128-byte FP32 stores per warp
// and row).
// Off-band tiles hold no diagonal entry; entries in padding rows or columns
// are 0.
template <bool GENERAL>
__global__ void __launch_bounds__(256)
k_matern_tiles_df(const double *__restrict__ X, const double *__restrict__ Y, int64_t n, Tiles tl,
                  const __grid_constant__ egs_matern_df Dg, const __grid_constant__ egs_matern_params Pg,
                  const float2 *__restrict__ ctab_g)
{
    __shared__ float etab[2 * EGS_DF_TAB];
    __shared__ float2 ctab[GENERAL ? EGS_MT_DOUBLES : 1];
    __shared__ float4 rows[1024];
    const int b = tl.b;
    int ri, tj;
    tile_decode((int64_t)blockIdx.x, ri, tj);
    const int ti = ri + tl.band;
    for (int i = threadIdx.x; i < 2 * EGS_DF_TAB; i += blockDim.x) etab[i] = Dg.tab[i];
    if (GENERAL)
        for (int i = threadIdx.x; i < EGS_MT_DOUBLES; i += blockDim.x) ctab[i] = ctab_g[i];
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
        const int64_t gi = (int64_t)ti * b + r;
        rows[r] = gi < n ? split_point(X[gi], Y[gi]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const df::Consts C{{Dg.inv_th2[0], Dg.inv_th2[1]}, Dg.kind};
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int c = (int)blockIdx.y * 64 + tx;
    const int64_t gj = (int64_t)tj * b + c;
    const float4 pj = gj < n ? split_point(X[gj], Y[gj]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t rlim = n - (int64_t)ti * b;  // rows r < rlim are real locations
    float *t32 = tl.t32(ti, tj) + c;
    for (int r = ty; r < b; r += 4) {
        df::F2 v{0.0f, 0.0f};
        if (r < rlim && gj < n) v = df::matern_entry_df<GENERAL>(C, rows[r], pj, etab, ctab, &Pg);
        const size_t off = (size_t)r * b;
        t32[off] = v.h;
    }
}

// The general-nu local polynomials split into float pairs (hi, lo).
__global__ void k_split_table(const double *__restrict__ tab, float2 *__restrict__ out)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i < EGS_MT_DOUBLES) {
        const double v = tab[i];
        const float h = __double2float_rn(v);
        out[i] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

// The local polynomials of a general nu: one warp per sub-interval.
__global__ void __launch_bounds__(256) k_matern_table(const __grid_constant__ egs_matern_params Pg, double *tab)
{
    __shared__ egs_matern_params Ps;
    __shared__ double vals[8][EGS_MT_NC];
    stage_params(&Pg, &Ps);
    const int w = threadIdx.x >> 5;
    const int iv = (int)blockIdx.x * 8 + w;
    if (iv < EGS_MT_OCT * EGS_MT_SUB) matern_table_interval(&Ps, iv, tab, vals[w]);
}

bool matern_df_applies(const egs_matern_params &P, bool have_table, egs_matern_df *D)
{
    if (P.metric != EGS_DIST_EUCLIDEAN) return false;
    if (P.kind == EGS_MATERN_GENERAL && !have_table) return false;
    return egs_matern_df_init(&P, D) == 0;
}

float2 *matern_df_table(double *tab) { return reinterpret_cast<float2 *>(tab + EGS_MT_DOUBLES); }

cudaError_t launch_matern_table(const egs_matern_params &P, double *tab, cudaStream_t s, KernelTimer *kt)
{
    constexpr int blocks = (EGS_MT_OCT * EGS_MT_SUB + 7) / 8;
    EGS_LAUNCH(kt, KC_GEN, s, k_matern_table<<<blocks, 256, 0, s>>>(P, tab));
    return cudaGetLastError();
}

cudaError_t launch_matern_tiles(const double *X, const double *Y, int64_t n, const Tiles &tl,
                                const egs_matern_params &P, cudaStream_t s, KernelTimer *kt, double *tab)
{
    const double *t = nullptr;
    if (tab && P.kind == EGS_MATERN_GENERAL) {
        cudaError_t e = launch_matern_table(P, tab, s, kt);
        if (e != cudaSuccess) return e;
        t = tab;
    }
    const unsigned nsub = (unsigned)((tl.b / 64) * (tl.b / 64));
    egs_matern_df D;
    if (!tl.dense() && matern_df_applies(P, tab != nullptr, &D)) {
        // mixed layout: FP64 band tiles directly, the FP32 off-band tiles in
        // double-float
        EGS_LAUNCH(kt, KC_GEN, s,
                   k_matern_tiles<<<dim3((unsigned)(tl.T * tl.band), nsub), 256, 0, s>>>(X, Y, n, tl, P, t, 1));
        const dim3 grid((unsigned)Tiles::f32_tiles(tl.T, tl.band), (unsigned)(tl.b / 64));
        if (P.kind == EGS_MATERN_GENERAL) {
            float2 *ctab = matern_df_table(tab);
            EGS_LAUNCH(kt, KC_GEN, s, k_split_table<<<(EGS_MT_DOUBLES + 255) / 256, 256, 0, s>>>(tab, ctab));
            EGS_LAUNCH(kt, KC_GEN, s, k_matern_tiles_df<true><<<grid, 256, 0, s>>>(X, Y, n, tl, D, P, ctab));
        } else {
            EGS_LAUNCH(kt, KC_GEN, s, k_matern_tiles_df<false><<<grid, 256, 0, s>>>(X, Y, n, tl, D, P, nullptr));
        }
        return cudaGetLastError();
    }
    const size_t ntiles = (size_t)tl.T * (tl.T + 1) / 2;
    EGS_LAUNCH(kt, KC_GEN, s, k_matern_tiles<<<dim3((unsigned)ntiles, nsub), 256, 0, s>>>(X, Y, n, tl, P, t, 0));
    return cudaGetLastError();
}

cudaError_t launch_matern_tiles_f64(const double *X, const double *Y, const TileGeom &g,
                                    const egs_matern_params &P, double *tiles, cudaStream_t s, KernelTimer *kt,
                                    double *tab)
{
    const Tiles tl{tiles, nullptr, g.b, g.T, g.T};
    return launch_matern_tiles(X, Y, g.n, tl, P, s, kt, tab);
}

}  // namespace egs
