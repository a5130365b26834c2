// Per-cell quantities and combining rules shared by the reduction kernels.
#pragma once

#include <math.h>

#include "stencil.cuh"

namespace ac {

template <typename T>
struct PtrPack {
    T *p[NF];
};

__device__ __forceinline__ double red_init(int op) {
    return op == AC_MAX ? -INFINITY : (op == AC_MIN ? INFINITY : 0.0);
}

__device__ __forceinline__ double red_combine(int op, double a, double b) {
    if (op == AC_MAX) return fmax(a, b);
    if (op == AC_MIN) return fmin(a, b);
    return a + b;
}

template <typename R, class IX>
__device__ double cell_quantity(const R *const *f, const IX &ix, const DevCoefs<R> &k,
                                int quantity) {
    const long long c0 = ix(0, 0, 0);
    if (quantity < NF) return (double)ldg(f[quantity] + c0);
    const double ux = ldg(f[1] + c0), uy = ldg(f[2] + c0), uz = ldg(f[3] + c0);
    const double u2 = ux * ux + uy * uy + uz * uz;
    if (quantity == AC_Q_UMAG) return sqrt(u2);
    const double lnrho = ldg(f[0] + c0);
    if (quantity == AC_Q_EKIN) return 0.5 * exp(lnrho) * u2;
    // B = curl A with the first-derivative operator, evaluated in binary64.
    const double Bx = (double)op_d1<1>(f[7], ix, k.d1[1]) - (double)op_d1<2>(f[6], ix, k.d1[2]);
    const double By = (double)op_d1<2>(f[5], ix, k.d1[2]) - (double)op_d1<0>(f[7], ix, k.d1[0]);
    const double Bz = (double)op_d1<0>(f[6], ix, k.d1[0]) - (double)op_d1<1>(f[5], ix, k.d1[1]);
    const double b2 = Bx * Bx + By * By + Bz * Bz;
    if (quantity == AC_Q_EMAG) return 0.5 * b2;
    // AC_Q_CFL
    const double ss = ldg(f[4] + c0);
    const double cs2 = (double)k.cs2_ref * exp((double)k.gamma_cp * ss + (double)k.gm1 * lnrho);
    return sqrt(u2) + sqrt(cs2 + b2 * exp(-lnrho));
}

}  // namespace ac
