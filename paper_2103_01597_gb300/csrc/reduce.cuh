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

// Per-cell quantity, evaluated in the field precision R (binary64 fields: all
// in binary64) and widened to binary64 for the accumulation.
template <typename R, class IX, int RAD = 3>
__device__ double cell_quantity(const R *const *f, const IX &ix, const DevCoefs<R> &k,
                                int quantity) {
    const long long c0 = ix(0, 0, 0);
    if (quantity < NF) return (double)ldg(f[quantity] + c0);
    const R ux = ldg(f[1] + c0), uy = ldg(f[2] + c0), uz = ldg(f[3] + c0);
    const R u2 = ux * ux + uy * uy + uz * uz;
    if (quantity == AC_Q_UMAG) return (double)sqrt(u2);
    const R lnrho = ldg(f[0] + c0);
    if (quantity == AC_Q_EKIN) return (double)((R)0.5 * exp(lnrho) * u2);
    // B = curl A with the first-derivative operator.
    const GlobalView<R, IX> ax{f[5], ix}, ay{f[6], ix}, az{f[7], ix};
    const R Bx = op_d1<1, RAD>(az, k.d1[1]) - op_d1<2, RAD>(ay, k.d1[2]);
    const R By = op_d1<2, RAD>(ax, k.d1[2]) - op_d1<0, RAD>(az, k.d1[0]);
    const R Bz = op_d1<0, RAD>(ay, k.d1[0]) - op_d1<1, RAD>(ax, k.d1[1]);
    const R b2 = Bx * Bx + By * By + Bz * Bz;
    if (quantity == AC_Q_EMAG) return (double)((R)0.5 * b2);
    // AC_Q_CFL
    const R ss = ldg(f[4] + c0);
    const R cs2 = k.cs2_ref * exp(k.gamma_cp * ss + k.gm1 * lnrho);
    return (double)(sqrt(u2) + sqrt(cs2 + b2 * exp(-lnrho)));
}

}  // namespace ac
