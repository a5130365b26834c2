// Device-side stencil machinery: cell indexing with the periodic map of
// Sec. 3.3 or a radius-3 halo, the central operators of order 2r on the point
// set of Sec. 4 Eq. 13 (r = 3 there; r = 1, 2, 4 widen it), and the fused RHS
// (Eqs. B.1-B.4) + Runge-Kutta update of one cell.
#pragma once

#include <cuda_runtime.h>

#include "ac_internal.h"
#include "bounds.cuh"
#include "exp_table.cuh"

namespace ac {

// Coefficients and constants in the kernel's arithmetic type R.
template <typename R>
struct DevCoefs {
    R d1[3][MAX_RADIUS];
    R d2[3][MAX_RADIUS + 1];
    R dc[3][MAX_RADIUS];
    R nu, eta, nu3, two_nu;  // nu3: coefficient of grad(div u), nu / 3 + zeta; 2 nu
    R inv_cp, cs2_ref, gamma_cp, gm1, cp_gm1;
    R inv_T_ref;             // c_p (gamma - 1) / cs2_ref
    R K, zeta, hc;           // conduction, bulk viscosity, H - C (Eqs. B.2-B.3)
};

template <typename R>
inline DevCoefs<R> to_dev(const StencilCoefs &c, const PhysConsts &p) {
    DevCoefs<R> d;
    for (int a = 0; a < 3; ++a) {
        for (int m = 0; m < MAX_RADIUS; ++m) {
            d.d1[a][m] = (R)c.d1[a][m];
            d.dc[a][m] = (R)c.dc[a][m];
        }
        for (int m = 0; m <= MAX_RADIUS; ++m) d.d2[a][m] = (R)c.d2[a][m];
    }
    d.nu = (R)p.nu;
    d.eta = (R)p.eta;
    d.nu3 = (R)(p.nu / 3.0 + p.zeta);
    d.two_nu = (R)(2.0 * p.nu);
    d.inv_cp = (R)p.inv_cp;
    d.cs2_ref = (R)p.cs2_ref;
    d.gamma_cp = (R)p.gamma_cp;
    d.gm1 = (R)p.gm1;
    d.cp_gm1 = (R)p.cp_gm1;
    d.inv_T_ref = (R)(p.cp_gm1 / p.cs2_ref);
    d.K = (R)p.K;
    d.zeta = (R)p.zeta;
    d.hc = (R)p.hc;
    return d;
}

// Periodic wrap of an index that is at most MAX_RADIUS cells outside [0, n).
__device__ __forceinline__ int wrap_near(int v, int n) {
    // n >= 1; v in [-MAX_RADIUS, n + MAX_RADIUS - 1]
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// Cell addressing without a halo: every offset is wrapped (Sec. 3.3 map);
// offsets up to RAD cells along each axis.  OFF is the type of the stored row
// and plane offsets: 32-bit ones (arrays of fewer than 2^31 elements) save
// fourteen registers per thread, which the register-bound kernels feel.
template <int RAD, typename OFF = long long>
struct IdxPeriodicR {
    static constexpr int W = 2 * RAD + 1;
    int xo[W];
    OFF yo[W];
    OFF zo[W];
    AC_BC_ONLY(long long bc_lim;)
    __device__ __forceinline__ void set_xy(int i, int j, const Geom &g) {
        AC_BC_ONLY(bc_lim = g.elems;)
#pragma unroll
        for (int d = 0; d < W; ++d) {
            xo[d] = wrap_near(i + d - RAD, g.nx);
            yo[d] = (OFF)wrap_near(j + d - RAD, g.ny) * (OFF)g.px;
        }
    }
    __device__ __forceinline__ void set_z(int k, const Geom &g) {
#pragma unroll
        for (int d = 0; d < W; ++d) zo[d] = (OFF)wrap_near(k + d - RAD, g.nz) * (OFF)g.pxy;
    }
    __device__ __forceinline__ void set_x(int i, const Geom &g) {
#pragma unroll
        for (int d = 0; d < W; ++d) xo[d] = wrap_near(i + d - RAD, g.nx);
    }
    __device__ __forceinline__ long long operator()(int dx, int dy, int dz) const {
        return AC_BC((long long)(zo[dz + RAD] + yo[dy + RAD] + xo[dx + RAD]), bc_lim, AC_BC_STENCIL);
    }
};
using IdxPeriodic = IdxPeriodicR<3>;
using IdxPeriodic32 = IdxPeriodicR<3, int>;  // arrays of fewer than 2^31 elements

// Cell addressing inside a padded array whose halo holds the periodic images.
struct IdxPadded {
    long long c;     // current cell
    long long jrow;  // origin + j * px
    long long row;   // jrow + k * pxy
    int i, px;
    long long pxy;
    AC_BC_ONLY(long long bc_lim;)
    __device__ __forceinline__ void set_xy(int i_, int j, const Geom &g) {
        AC_BC_ONLY(bc_lim = g.elems;)
        px = g.px;
        pxy = g.pxy;
        i = i_;
        jrow = g.origin + (long long)j * g.px;
        row = jrow;
        c = row + i;
    }
    __device__ __forceinline__ void set_z(int k, const Geom &) {
        row = jrow + (long long)k * pxy;
        c = row + i;
    }
    __device__ __forceinline__ void set_x(int i_, const Geom &) {
        i = i_;
        c = row + i;
    }
    __device__ __forceinline__ long long operator()(int dx, int dy, int dz) const {
        return AC_BC(c + dz * pxy + (long long)dy * px + dx, bc_lim, AC_BC_STENCIL);
    }
};

template <typename R>
__device__ __forceinline__ R ldg(const R *p) { return __ldg(p); }

// ---- field views -----------------------------------------------------------
// A view returns one field's value at offset (dx, dy, dz) from the current cell;
// the offsets are compile-time constants after unrolling.

// Global memory through the read-only path, addressed by IX.
template <typename R, class IX>
struct GlobalView {
    const R *__restrict__ f;
    const IX &ix;
    __device__ __forceinline__ R operator()(int dx, int dy, int dz) const {
        return ldg(f + ix(dx, dy, dz));
    }
};

// All eight fields of one cell in global memory.
template <typename R, class IX>
struct GlobalCell {
    const R *const *f;
    const IX &ix;
    __device__ __forceinline__ GlobalView<R, IX> operator[](int q) const { return {f[q], ix}; }
    __device__ __forceinline__ long long center() const { return ix(0, 0, 0); }
};

// ---- central operators of order 2 RAD (RAD = 3: sixth order, Sec. 4) ------
// Sums run m = 1 .. RAD in that order, so RAD = 3 rounds exactly as the
// sixth-order formulas written out term by term.

// First derivative along axis AX: sum_m d1[m-1] (f_m - f_-m).
template <int AX, int RAD = 3, typename R, class V>
__device__ __forceinline__ R op_d1(const V &f, const R (&c)[MAX_RADIUS]) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    R sum = c[0] * (f(ox, oy, oz) - f(-ox, -oy, -oz));
#pragma unroll
    for (int m = 2; m <= RAD; ++m)
        sum += c[m - 1] * (f(m * ox, m * oy, m * oz) - f(-m * ox, -m * oy, -m * oz));
    return sum;
}

// Second derivative along axis AX: d2[0] f_0 + sum_m d2[m] (f_m + f_-m).
template <int AX, int RAD = 3, typename R, class V>
__device__ __forceinline__ R op_d2(const V &f, R f0, const R (&c)[MAX_RADIUS + 1]) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    R sum = c[0] * f0;
#pragma unroll
    for (int m = 1; m <= RAD; ++m)
        sum += c[m] * (f(m * ox, m * oy, m * oz) + f(-m * ox, -m * oy, -m * oz));
    return sum;
}

// Mixed derivative in the plane of axes A < B from the face diagonals of Eq. 13:
// sum_m dc[m-1] S_m, S_m = f(+m,+m) + f(-m,-m) - f(+m,-m) - f(-m,+m).
template <int A, int B, int RAD = 3, typename R, class V>
__device__ __forceinline__ R op_dab(const V &f, const R (&c)[MAX_RADIUS]) {
    constexpr int ax = A == 0, ay = A == 1, az = A == 2;
    constexpr int bx = B == 0, by = B == 1, bz = B == 2;
    R S[RAD];
#pragma unroll
    for (int m = 1; m <= RAD; ++m) {
        const R pp = f(m * (ax + bx), m * (ay + by), m * (az + bz));
        const R mm = f(-m * (ax + bx), -m * (ay + by), -m * (az + bz));
        const R pm = f(m * (ax - bx), m * (ay - by), m * (az - bz));
        const R mp = f(-m * (ax - bx), -m * (ay - by), -m * (az - bz));
        S[m - 1] = (pp + mm) - (pm + mp);
    }
    R sum = c[0] * S[0];
#pragma unroll
    for (int m = 2; m <= RAD; ++m) sum += c[m - 1] * S[m - 1];
    return sum;
}

// Plane index of the axis pair (a, b): xy -> 0, xz -> 1, yz -> 2.
template <int A, int B>
struct Plane {
    static constexpr int lo = A < B ? A : B;
    static constexpr int hi = A < B ? B : A;
    static constexpr int id = lo == 0 ? (hi == 1 ? 0 : 1) : 2;
};

// Second derivatives of one vector component V_C: its Laplacian, the pure
// derivative along its own axis (d_CC V_C) and the two mixed derivatives
// d_C d_b V_C (b != C) that enter grad(div V).
template <int C, int RAD = 3, typename R, class V>
__device__ __forceinline__ void component_second(const V &f, R f0, const DevCoefs<R> &k, R &lap,
                                                 R &dcc, R &cross_b1, R &cross_b2) {
    const R dxx = op_d2<0, RAD>(f, f0, k.d2[0]);
    const R dyy = op_d2<1, RAD>(f, f0, k.d2[1]);
    const R dzz = op_d2<2, RAD>(f, f0, k.d2[2]);
    lap = dxx + dyy + dzz;
    constexpr int B1 = C == 0 ? 1 : 0;
    constexpr int B2 = C == 2 ? 1 : 2;
    dcc = C == 0 ? dxx : (C == 1 ? dyy : dzz);
    cross_b1 = op_dab<(C < B1 ? C : B1), (C < B1 ? B1 : C), RAD>(f, k.dc[Plane<C, B1>::id]);
    cross_b2 = op_dab<(C < B2 ? C : B2), (C < B2 ? B2 : C), RAD>(f, k.dc[Plane<C, B2>::id]);
}

template <typename R> __device__ __forceinline__ R dev_exp(R x);
template <> __device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }

// ---- binary64 exp by Tang's table-driven method (ACM TOMS 15(2), 1989) ------
// x = N ln2/256 + r with N = rint(256 x / ln 2) and |r| <= ln2/512; with
// N = 256 m + j, exp(x) = 2^m 2^(j/256) exp(r), exp(r) - 1 from its degree-4
// Taylor polynomial (truncation below 4e-17 relative).  The same reduction gives
// exp(-x) from 2^(-j/256) and exp(-r).  Measured on GB300 in FP64-pipe DFMA
// equivalents: 8.7 for exp alone and 13.4 for the pair, against 15.0 for CUDA's
// exp and 7.5 for a division; within 1 ulp of CUDA's exp for |x| < 700.  `tab` is
// EXP_TAB (exp_table.cuh) staged in shared memory.

// |x| < 700 (finite, and every result below stays normal), tested on the bits.
__device__ __forceinline__ bool exp_tab_ok(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffll) < 0x4085e00000000000ll;  // 700.0
}

struct ExpReduced {
    double r;
    int n;
};

__device__ __forceinline__ ExpReduced exp_reduce(double x) {
    constexpr double SH = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
    const double t = fma(x, EXP_INV, SH);
    const double nd = t - SH;
    ExpReduced e;
    e.n = (int)(__double_as_longlong(t) & 0xffffffffll);  // low word of t = N (two's complement)
    e.r = fma(-nd, EXP_L2, fma(-nd, EXP_L1, x));          // nd * EXP_L1 is exact
    return e;
}

// 2^m y for normal y and a normal result: m added to the exponent field.
__device__ __forceinline__ double exp_scale(double y, int m) {
    return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
}

__device__ __forceinline__ double exp_tab(double x, const double *tab) {
    const ExpReduced e = exp_reduce(x);
    double p = fma(e.r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, e.r, 0.5);
    p = fma(p * e.r, e.r, e.r);  // exp(r) - 1
    const double tj = tab[e.n & 255];
    return exp_scale(fma(tj, p, tj), e.n >> 8);
}

__device__ __forceinline__ void exp_tab_pm(double x, const double *tab, double &ep, double &em) {
    const ExpReduced e = exp_reduce(x);
    double p = fma(e.r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, e.r, 0.5);
    p = fma(p * e.r, e.r, e.r);  // exp(r) - 1
    double q = fma(e.r, 1.0 / 24.0, -1.0 / 6.0);
    q = fma(q, e.r, 0.5);
    q = fma(q * e.r, e.r, -e.r);  // exp(-r) - 1
    const int j = e.n & 255, m = e.n >> 8;
    const double tp = tab[j], tm = tab[256 + j];
    ep = exp_scale(fma(tp, p, tp), m);
    em = exp_scale(fma(tm, q, tm), -m);
}

// Copy EXP_TAB into the shared array `tab` (every thread of the CTA calls this;
// it ends with a barrier).
__device__ __forceinline__ void exp_tab_stage(double *tab) {
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    for (int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x; t < 512;
         t += nt)
        tab[t] = EXP_TAB[t];
    __syncthreads();
}

// The thermodynamic factors with CUDA's exp and a division.  (Kept inline: out
// of line, the call made the binary64 substep-0 kernel 13% slower through
// register allocation, although it is never taken on physical states.)
template <typename R>
__device__ __forceinline__ void thermo_lib(R lnrho, R xi, R cs2_ref, R cp_gm1, R &rho_inv, R &cs2,
                                           R &inv_T) {
    rho_inv = dev_exp<R>(-lnrho);
    cs2 = cs2_ref * dev_exp<R>(xi);
    inv_T = cp_gm1 / cs2;
}

// Thermodynamic factors of one cell: c_s^2 = c_s0^2 exp(gamma s / c_p + (gamma-1)
// (ln rho - ln rho0)) = cs2_ref exp(xi) with xi = gamma s / c_p + (gamma-1) ln rho
// and cs2_ref = c_s0^2 exp(-(gamma-1) ln rho0); 1/rho = exp(-ln rho); 1/T =
// c_p (gamma - 1) / c_s^2 = inv_T_ref exp(-xi).  With `etab` (binary64 only) the
// exponentials come from the table-driven exp above and 1/T from exp(-xi) instead
// of a division.
template <typename R>
struct Thermo {
    R rho_inv, cs2, inv_T;
};

template <typename R>
__device__ __forceinline__ Thermo<R> thermo_factors(R lnrho, R ss, const DevCoefs<R> &k,
                                                    const double *etab) {
    const R xi = k.gamma_cp * ss + k.gm1 * lnrho;
    Thermo<R> t;
    if (sizeof(R) != 8 || etab == nullptr) {
        thermo_lib<R>(lnrho, xi, k.cs2_ref, k.cp_gm1, t.rho_inv, t.cs2, t.inv_T);
    } else if (exp_tab_ok((double)lnrho) && exp_tab_ok((double)xi)) {
        t.rho_inv = (R)exp_tab(-(double)lnrho, etab);
        double ep, em;
        exp_tab_pm((double)xi, etab, ep, em);
        t.cs2 = k.cs2_ref * (R)ep;
        t.inv_T = k.inv_T_ref * (R)em;
    } else {
        thermo_lib<R>(lnrho, xi, k.cs2_ref, k.cp_gm1, t.rho_inv, t.cs2, t.inv_T);
    }
    return t;
}

// Eqs. B.1-B.4 at one cell (mu0 = 1) given the centre values and the derivative
// terms: gl, gs, gu[m][a] first derivatives of ln rho, s, u_m; B = curl A;
// viscl = nu lap u + (nu / 3 + zeta) grad(div u) (the bulk viscosity of Eq. B.2
// folded into the grad-div coefficient); lapa = lap A; J = grad(div A) - lap A.
// The forcing term `frc` is added to du/dt.  EXT adds the remaining terms of
// Eq. B.3: H - C, zeta rho (div u)^2 and div(K grad T) (from lapxi = lap xi);
// without EXT they are zero.  `th` holds the cell's thermodynamic factors.
// Output order: Table B.1.
template <typename R, bool EXT = false>
__device__ __forceinline__ void cell_physics(R lnrho, const R (&u)[3], R ss, const R (&gl)[3],
                                             const R (&gs)[3], const R (&gu)[3][3],
                                             const R (&B)[3], const R (&viscl)[3],
                                             const R (&lapa)[3], const R (&J)[3],
                                             const DevCoefs<R> &k, const R frc[3], R out[NF],
                                             R *cfl, R lapxi, const Thermo<R> &th) {
    const R rho_inv = th.rho_inv, cs2 = th.cs2, inv_T = th.inv_T;

    const R divu = gu[0][0] + gu[1][1] + gu[2][2];
    const R third_div = divu * (R)(1.0 / 3.0);


    // Traceless rate of strain S.
    const R Sxx = gu[0][0] - third_div, Syy = gu[1][1] - third_div, Szz = gu[2][2] - third_div;
    const R Sxy = (R)0.5 * (gu[0][1] + gu[1][0]);
    const R Sxz = (R)0.5 * (gu[0][2] + gu[2][0]);
    const R Syz = (R)0.5 * (gu[1][2] + gu[2][1]);
    const R SS2 = Sxx * Sxx + Syy * Syy + Szz * Szz + (R)2 * (Sxy * Sxy + Sxz * Sxz + Syz * Syz);
    const R SG[3] = {Sxx * gl[0] + Sxy * gl[1] + Sxz * gl[2],
                     Sxy * gl[0] + Syy * gl[1] + Syz * gl[2],
                     Sxz * gl[0] + Syz * gl[1] + Szz * gl[2]};

    const R JxB[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2],
                      J[0] * B[1] - J[1] * B[0]};
    const R UxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2],
                      u[0] * B[1] - u[1] * B[0]};
    const R J2 = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];

    // Eq. B.1
    out[0] = -(u[0] * gl[0] + u[1] * gl[1] + u[2] * gl[2]) - divu;
    // Eq. B.2
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const R adv = u[0] * gu[m][0] + u[1] * gu[m][1] + u[2] * gu[m][2];
        const R press = cs2 * (gs[m] * k.inv_cp + gl[m]);
        const R visc = viscl[m] + k.two_nu * SG[m];
        out[1 + m] = (visc - adv) - press + JxB[m] * rho_inv + frc[m];
    }
    // Eq. B.3: Ds/Dt = (eta j^2 + 2 rho nu S:S) / (rho T)
    out[4] = -(u[0] * gs[0] + u[1] * gs[1] + u[2] * gs[2])
           + (k.eta * J2 * rho_inv + k.two_nu * SS2) * inv_T;
    if (EXT) {
        // + (H - C + zeta rho (div u)^2) / (rho T) + div(K grad T) / (rho T), the last
        // = K (lap xi + |grad xi|^2) / rho with xi = gamma s / c_p + (gamma-1) ln rho
        // (grad T = T grad xi); lapxi is passed in, grad xi built from gs and gl.
        R gxi2 = (R)0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const R gxi = k.gamma_cp * gs[m] + k.gm1 * gl[m];
            gxi2 += gxi * gxi;
        }
        out[4] += (k.hc * rho_inv + k.zeta * divu * divu) * inv_T + k.K * rho_inv * (lapxi + gxi2);
    }
    // Eq. B.4
#pragma unroll
    for (int m = 0; m < 3; ++m) out[5 + m] = UxB[m] + k.eta * lapa[m];
    if (cfl) {
        const R b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        const R u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        *cfl = sqrt(u2) + sqrt(cs2 + b2 * rho_inv);
    }
}


// The same with the thermodynamic factors computed at its top by CUDA's exp and
// a division, in the statement order the binary64 direct-load kernels were
// measured with (their register allocation depends on it).
template <typename R, bool EXT = false>
__device__ __forceinline__ void cell_physics(R lnrho, const R (&u)[3], R ss, const R (&gl)[3],
                                             const R (&gs)[3], const R (&gu)[3][3],
                                             const R (&B)[3], const R (&viscl)[3],
                                             const R (&lapa)[3], const R (&J)[3],
                                             const DevCoefs<R> &k, const R frc[3], R out[NF],
                                             R *cfl, R lapxi) {
    const R rho_inv = dev_exp<R>(-lnrho);
    const R cs2 = k.cs2_ref * dev_exp<R>(k.gamma_cp * ss + k.gm1 * lnrho);
    const R inv_T = k.cp_gm1 / cs2;
    cell_physics<R, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, k, frc, out, cfl, lapxi,
                         Thermo<R>{rho_inv, cs2, inv_T});
}


// `f` is a cell accessor: f[q] is the view of field q around the cell.  With
// `cfl` non-null, the fastest signal speed of the input state at the cell,
// |u| + sqrt(c_s^2 + |B|^2 / rho) (mu0 = 1), is written there as well.
template <typename R, int RAD = 3, bool EXT = false, class CELL>
__device__ __forceinline__ void cell_rhs(const CELL &f, const DevCoefs<R> &k, const R frc[3],
                                         R out[NF], R *cfl = nullptr) {
    const R lnrho = f[0](0, 0, 0);
    const R u[3] = {f[1](0, 0, 0), f[2](0, 0, 0), f[3](0, 0, 0)};
    const R ss = f[4](0, 0, 0);
    const R aa[3] = {f[5](0, 0, 0), f[6](0, 0, 0), f[7](0, 0, 0)};

    // First derivatives.
    R gl[3], gs[3], gu[3][3], ga[3][3];
    gl[0] = op_d1<0, RAD>(f[0], k.d1[0]);
    gl[1] = op_d1<1, RAD>(f[0], k.d1[1]);
    gl[2] = op_d1<2, RAD>(f[0], k.d1[2]);
    gs[0] = op_d1<0, RAD>(f[4], k.d1[0]);
    gs[1] = op_d1<1, RAD>(f[4], k.d1[1]);
    gs[2] = op_d1<2, RAD>(f[4], k.d1[2]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        gu[m][0] = op_d1<0, RAD>(f[1 + m], k.d1[0]);
        gu[m][1] = op_d1<1, RAD>(f[1 + m], k.d1[1]);
        gu[m][2] = op_d1<2, RAD>(f[1 + m], k.d1[2]);
        ga[m][0] = op_d1<0, RAD>(f[5 + m], k.d1[0]);
        ga[m][1] = op_d1<1, RAD>(f[5 + m], k.d1[1]);
        ga[m][2] = op_d1<2, RAD>(f[5 + m], k.d1[2]);
    }

    // Second derivatives: Laplacians and grad(div .) of u and A.
    R lapu[3], lapa[3], gdu[3], gda[3];
    {
        R dcc, c1, c2;
        component_second<0, RAD>(f[1], u[0], k, lapu[0], dcc, c1, c2);  // c1 = d_xy u_x, c2 = d_xz u_x
        gdu[0] = dcc;
        gdu[1] = c1;
        gdu[2] = c2;
        component_second<1, RAD>(f[2], u[1], k, lapu[1], dcc, c1, c2);  // c1 = d_xy u_y, c2 = d_yz u_y
        gdu[0] += c1;
        gdu[1] += dcc;
        gdu[2] += c2;
        component_second<2, RAD>(f[3], u[2], k, lapu[2], dcc, c1, c2);  // c1 = d_xz u_z, c2 = d_yz u_z
        gdu[0] += c1;
        gdu[1] += c2;
        gdu[2] += dcc;
    }
    {
        R dcc, c1, c2;
        component_second<0, RAD>(f[5], aa[0], k, lapa[0], dcc, c1, c2);
        gda[0] = dcc;
        gda[1] = c1;
        gda[2] = c2;
        component_second<1, RAD>(f[6], aa[1], k, lapa[1], dcc, c1, c2);
        gda[0] += c1;
        gda[1] += dcc;
        gda[2] += c2;
        component_second<2, RAD>(f[7], aa[2], k, lapa[2], dcc, c1, c2);
        gda[0] += c1;
        gda[1] += c2;
        gda[2] += dcc;
    }

    // B = curl A, j = grad(div A) - lap A, nu (lap u + grad(div u) / 3).
    const R B[3] = {ga[2][1] - ga[1][2], ga[0][2] - ga[2][0], ga[1][0] - ga[0][1]};
    const R J[3] = {gda[0] - lapa[0], gda[1] - lapa[1], gda[2] - lapa[2]};
    R viscl[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) viscl[m] = k.nu * lapu[m] + k.nu3 * gdu[m];
    R lapxi = (R)0;
    if (EXT) {  // lap xi = gamma / c_p lap s + (gamma - 1) lap ln rho
        const R lsx = op_d2<0, RAD>(f[4], ss, k.d2[0]), lsy = op_d2<1, RAD>(f[4], ss, k.d2[1]),
                lsz = op_d2<2, RAD>(f[4], ss, k.d2[2]);
        const R llx = op_d2<0, RAD>(f[0], lnrho, k.d2[0]), lly = op_d2<1, RAD>(f[0], lnrho, k.d2[1]),
                llz = op_d2<2, RAD>(f[0], lnrho, k.d2[2]);
        lapxi = k.gamma_cp * (lsx + lsy + lsz) + k.gm1 * (llx + lly + llz);
    }
    // binary32: factors computed before the call (ptxas then gives the r = 1
    // substep-0 kernel 96 instead of 114 registers, measured 19.5 -> 20.2
    // Gcell-updates/s at 512^3); binary64: at the top of the physics, the order
    // its direct-load kernels were measured with
    if constexpr (sizeof(R) == 4)
        cell_physics<R, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, k, frc, out, cfl, lapxi,
                             thermo_factors<R>(lnrho, ss, k, nullptr));
    else
        cell_physics<R, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, k, frc, out, cfl, lapxi);
}

// Block-wide max of a non-negative value folded into a global 64-bit word that
// holds the bits of a binary64 (ordered like the values for non-negative
// numbers; NaN bits compare above every finite value).
__device__ __forceinline__ void block_max_to_global(double v, unsigned long long *gmax) {
    __shared__ unsigned long long bmax;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) bmax = 0ull;
    __syncthreads();
    unsigned long long bits = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((tid & 31) == 0) atomicMax(&bmax, bits);
    __syncthreads();
    if (tid == 0) atomicMax(gmax, bmax);
}

}  // namespace ac
