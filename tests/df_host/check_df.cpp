// CPU check of the double-float Matern evaluation of the mixed precisions
// (csrc/matern_df.cuh) against long double references: the error-free
// transformations are exact, and the closed forms stay within a few 1e-14 of
// theta1 (relative error about 1e-14 for x < 1).  Prints one line of
// key=value pairs.
#include <cstdio>
#include <cstdlib>
#include <random>

#include "cuda_shim.h"
#include "matern_df.cuh"

using namespace egs::df;
typedef long double ld;

static void split(ld v, float *h, float *l)
{
    const float a = (float)v;
    *h = a;
    *l = (float)(v - (ld)a);
}

int main()
{
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    // error-free transformations
    long bad_sum = 0, bad_prod = 0;
    for (int t = 0; t < 200000; ++t) {
        const float a = (float)((U(g) - 0.5) * std::exp2(40 * U(g) - 20));
        const float b = (float)((U(g) - 0.5) * std::exp2(40 * U(g) - 20));
        const F2 s = two_sum(a, b);
        if ((ld)s.h + (ld)s.l != (ld)a + (ld)b) ++bad_sum;
        const F2 p = two_prod(a, b);
        if ((ld)p.h + (ld)p.l != (ld)a * (ld)b) ++bad_prod;
    }
    // theta1 e^-x, (1 + x) e^-x, (1 + x + x^2/3) e^-x from split coordinates
    double worst_abs[3] = {0, 0, 0}, worst_rel_small[3] = {0, 0, 0};
    const double th1 = 1.7, th2 = 0.1;
    float tab[2 * EGS_DF_TAB];
    for (int j = 0; j < EGS_DF_TAB; ++j) split((ld)th1 * std::exp2((ld)-j / EGS_DF_TAB), &tab[2 * j], &tab[2 * j + 1]);
    for (int kind = 1; kind <= 3; ++kind) {
        Consts C;
        split(1.0L / (ld)th2, &C.inv_th2.h, &C.inv_th2.l);
        C.kind = kind;
        for (int t = 0; t < 200000; ++t) {
            const double xi = U(g), yi = U(g);
            const double near = (t % 3 == 0) ? 1e-3 : 1.0;
            const double xj = t % 3 == 0 ? xi + (U(g) - 0.5) * near : U(g);
            const double yj = t % 3 == 0 ? yi + (U(g) - 0.5) * near : U(g);
            float4 pi, pj;
            split(xi, &pi.x, &pi.y);
            split(yi, &pi.z, &pi.w);
            split(xj, &pj.x, &pj.y);
            split(yj, &pj.z, &pj.w);
            const F2 dx = diff(pi.x, pi.y, pj.x, pj.y), dy = diff(pi.z, pi.w, pj.z, pj.w);
            const F2 x = mul(sqrt_df(add(sqr(dx), sqr(dy))), C.inv_th2);
            const F2 v = matern_closed_df(C, x, tab);
            // reference from the same split coordinates
            const ld ddx = ((ld)pi.x + (ld)pi.y) - ((ld)pj.x + (ld)pj.y);
            const ld ddy = ((ld)pi.z + (ld)pi.w) - ((ld)pj.z + (ld)pj.w);
            const ld xr = std::sqrt(ddx * ddx + ddy * ddy) / (ld)th2;
            ld ref = (ld)th1 * std::exp(-xr);
            if (kind == 2) ref *= 1 + xr;
            if (kind == 3) ref *= 1 + xr + xr * xr / 3;
            const ld got = (ld)v.h + (ld)v.l;
            const double ea = (double)std::fabs((got - ref) / (ld)th1);
            if (ea > worst_abs[kind - 1]) worst_abs[kind - 1] = ea;
            if (xr < 1) {
                const double er = (double)std::fabs((got - ref) / ref);
                if (er > worst_rel_small[kind - 1]) worst_rel_small[kind - 1] = er;
            }
        }
    }
    std::printf("bad_sum=%ld bad_prod=%ld abs1=%.3e abs2=%.3e abs3=%.3e rel1=%.3e rel2=%.3e rel3=%.3e\n", bad_sum,
                bad_prod, worst_abs[0], worst_abs[1], worst_abs[2], worst_rel_small[0], worst_rel_small[1],
                worst_rel_small[2]);
    return 0;
}
