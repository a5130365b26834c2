// Binary64 substep with exact integer stencil sums (cubic periodic grids).
//
// GB300 executes two FP64 lanes per SM per cycle, so the binary64 substep is
// bound by its FP64 instruction count, most of which (about 400 of 600 per
// cell) are the additions and multiplications of the 54 stencils of Eq. 13.
// Here each field is first written as int64 fixed point about an offset of its
// own, F = round((f - c) 2^(50 - E)), with c the midpoint of the field's range
// and 2^E above its half-range, so |F| <= 2^50 + 2.  Every weight set of Eq. 13
// sums to zero, so the offset changes no derivative.  Every stencil numerator
// -- and every sum of numerators that share a coefficient (curl A, lap u,
// grad(div u), lap A, grad(div A)) -- is then an exact integer on the integer
// pipes (largest: 6744 |F| < 2^63), and only one int64 -> binary64 conversion
// and one multiplication per derivative term remain on the FP64 pipe.  The
// centre values used by the physics and the Runge-Kutta update are the
// binary64 state itself; the physics of Eqs. B.1-B.4 is unchanged binary64
// code (cell_physics).
//
// A plan kernel picks one of three modes per substep from the fields' ranges,
// on the device (no host round trip):
//  * FX_GROUP: the exponents E of the three components of u (and of A) lie
//    within one binade of each other, so they share the largest as one scale
//    (a component keeps at least 49 bits of its own range) and the
//    cross-component sums stay single integers;
//  * FX_FIELD: some component lies further below its group's largest, so every
//    field keeps its own scale and the cross-component sums (curl A,
//    grad(div u), grad(div A)) add per-field binary64 terms instead -- a
//    component far smaller than the others (a near-2-D flow, a weak field
//    component) is resolved to 2^-50 of its own range;
//  * FX_PLAIN: a NaN or infinity in the state, or a range outside
//    [2^-960, 2^960): the substep runs plain binary64 stencils, exactly what
//    AC_STENCIL_FP64 computes (so a non-finite value propagates as in the
//    definition and shows in the step's CFL word).
// The quantisation error of every stencil input is then at most half a unit
// of 2^(E - 49), E the field's own exponent: within a factor of about six of
// the worst-case binary64 rounding of the same stencil.
#pragma once

#include "substep.cuh"

namespace ac {

constexpr int FX_BITS = 50;
constexpr int FX_GROUP_SLACK = 1;  // binades a component may lie below its group's largest
enum { FX_GROUP = 0, FX_FIELD = 1, FX_PLAIN = 2 };

// Field -> group: 0 = ln rho, 1 = u, 2 = s, 3 = A.
__host__ __device__ __forceinline__ int fx_group(int q) {
    return q == 0 ? 0 : (q < 4 ? 1 : (q == 4 ? 2 : 3));
}

// Order-preserving map of binary64 bits to unsigned keys (NaNs sort beyond the
// infinities of their sign) and back.
__device__ __forceinline__ unsigned long long fx_key(unsigned long long b) {
    // negatives: every bit flipped; positives: the sign bit set
    return b ^ ((unsigned long long)((long long)b >> 63) | 0x8000000000000000ull);
}
__device__ __forceinline__ double fx_unkey(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// round(v 2^(FX_BITS - E)) modulo 2^64 for the binary64 v held in `b` (round
// half away from zero), by integer operations on the bits.  Two such values
// within 2^63 of each other subtract exactly in wrapping 64-bit arithmetic,
// however large each is.
__device__ __forceinline__ unsigned long long fx_round_grid(unsigned long long b, int E) {
    const int eb = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0xfffffffffffffull;
    int ex = -1074;
    if (eb != 0) {
        m |= 1ull << 52;
        ex = eb - 1075;
    }
    const int sh = ex + FX_BITS - E;  // |v| 2^(FX_BITS - E) = m 2^sh
    unsigned long long a;
    if (sh >= 0) {
        a = sh < 64 ? m << sh : 0ull;
    } else {
        const int k = -sh;
        a = k < 64 ? (m + (1ull << (k - 1))) >> k : 0ull;
    }
    return (b >> 63) ? 0ull - a : a;
}

struct FxPtrs {
    const double *f[NF];
    long long *F[NF];
};

// The quantisation plan of one substep (device memory, written by
// fx_plan_kernel, read by the quantisation and substep kernels).
struct FxPlan {
    int mode;                  // FX_GROUP, FX_FIELD or FX_PLAIN
    int zero[NF];              // constant field: F = 0
    int E[NF];                 // F = round((f - c) 2^(FX_BITS - E)); the scale is 2^(E - FX_BITS)
    unsigned long long C[NF];  // round(c 2^(FX_BITS - E)) modulo 2^64
    unsigned long long taken[3];  // substeps run in each mode (cumulative)
};

// Per-field extremes of the current state: stats[q] = largest key of field q,
// stats[NF + q] = its smallest key (the plan kernel resets both for the next
// substep).  Two cells per thread and iteration (16-byte loads; the arrays are
// 16-byte aligned), one CTA-wide reduction, then 16 atomics per CTA.
__global__ void __launch_bounds__(256) fx_stats_kernel(FxPtrs p, long long n,
                                                       unsigned long long *stats) {
    unsigned long long hi[NF], lo[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        hi[q] = 0ull;
        lo[q] = ~0ull;
    }
    const long long n2 = n >> 1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2;
         t += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p.f[q]) + t);
            const unsigned long long k0 = fx_key((unsigned long long)__double_as_longlong(v.x));
            const unsigned long long k1 = fx_key((unsigned long long)__double_as_longlong(v.y));
            const unsigned long long kh = k0 > k1 ? k0 : k1, kl = k0 > k1 ? k1 : k0;
            hi[q] = kh > hi[q] ? kh : hi[q];
            lo[q] = kl < lo[q] ? kl : lo[q];
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const unsigned long long k =
                fx_key((unsigned long long)__double_as_longlong(p.f[q][n - 1]));
            hi[q] = k > hi[q] ? k : hi[q];
            lo[q] = k < lo[q] ? k : lo[q];
        }
    }
    __shared__ unsigned long long red[2 * NF];
    if (threadIdx.x < NF) {
        red[threadIdx.x] = 0ull;
        red[NF + threadIdx.x] = ~0ull;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        unsigned long long a = hi[q], b = lo[q];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o);
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
            a = x > a ? x : a;
            b = y < b ? y : b;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&red[q], a);
            atomicMin(&red[NF + q], b);
        }
    }
    __syncthreads();
    if (threadIdx.x < NF)
        atomicMax(&stats[threadIdx.x], red[threadIdx.x]);
    else if (threadIdx.x < 2 * NF)
        atomicMin(&stats[threadIdx.x], red[threadIdx.x]);
}

// One warp: lane q < NF plans field q (offset, exponent), then the lanes agree
// on the mode.  Thread 0 also counts the substep under its mode.
__global__ void fx_plan_kernel(unsigned long long *stats, FxPlan *plan) {
    const int q = threadIdx.x;
    int bad = 0, zero = 1, e = -100000;
    double c = 0.0;
    if (q < NF) {
        const double hi = fx_unkey(stats[q]), lo = fx_unkey(stats[NF + q]);
        stats[q] = 0ull;        // ready for the next substep's extremes
        stats[NF + q] = ~0ull;
        if (!isfinite(hi) || !isfinite(lo)) {
            bad = 1;
        } else {
            c = 0.5 * lo + 0.5 * hi;
            const double r = fmax(hi - c, c - lo);
            if (r > 0.0) {
                zero = 0;
                if (!(r >= 0x1p-960 && r < 0x1p960))
                    bad = 1;
                else  // smallest E with r < 2^E
                    e = (int)((__double_as_longlong(r) >> 52) & 0x7ff) - 1022;
            }
        }
    }
    // largest exponent of the field's group over its non-constant members
    const int g = q < NF ? fx_group(q) : -1;
    int eg = -100000;
#pragma unroll
    for (int r = 0; r < NF; ++r) {
        const int er = __shfl_sync(0xffffffffu, e, r);
        if (fx_group(r) == g && er > eg) eg = er;
    }
    // group scales while every component's exponent is within one binade of its
    // group's largest (a component then keeps at least 49 bits of its own
    // range); a larger disparity takes per-field scales
    const int disparity = q < NF && !zero && e < eg - FX_GROUP_SLACK;
    const int any_bad = __any_sync(0xffffffffu, bad);
    const int any_disp = __any_sync(0xffffffffu, disparity);
    const int mode = any_bad ? FX_PLAIN : (any_disp ? FX_FIELD : FX_GROUP);
    if (q < NF) {
        int E = mode == FX_GROUP ? eg : e;
        const int valid = E > -100000;
        if (!valid) E = 0;
        plan->zero[q] = zero;
        plan->E[q] = E;
        plan->C[q] = fx_round_grid((unsigned long long)__double_as_longlong(c), E);
    }
    if (q == 0) {
        plan->mode = mode;
        plan->taken[mode] += 1ull;
    }
}

// F = round(f 2^(50 - E)) - round(c 2^(50 - E)) by integer operations on the
// binary64 bits; nothing to do in FX_PLAIN.  Two cells per thread and
// iteration (16-byte loads and stores: the int64 arrays have an even stride).
__global__ void __launch_bounds__(256) fx_quantize_kernel(FxPtrs p, long long n,
                                                          const FxPlan *plan) {
    if (plan->mode == FX_PLAIN) return;
    int E[NF], zero[NF];
    unsigned long long C[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        E[q] = plan->E[q];
        zero[q] = plan->zero[q];
        C[q] = plan->C[q];
    }
    const long long n2 = n >> 1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2;
         t += (long long)gridDim.x * blockDim.x) {
        // all eight loads ahead of the stores, so that they are in flight together
        double2 v[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) v[q] = __ldg(reinterpret_cast<const double2 *>(p.f[q]) + t);
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            longlong2 o;
            o.x = zero[q] ? 0ll
                          : (long long)(fx_round_grid((unsigned long long)__double_as_longlong(v[q].x),
                                                      E[q]) - C[q]);
            o.y = zero[q] ? 0ll
                          : (long long)(fx_round_grid((unsigned long long)__double_as_longlong(v[q].y),
                                                      E[q]) - C[q]);
            reinterpret_cast<longlong2 *>(p.F[q])[t] = o;
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(p.f[q][n - 1]);
            p.F[q][n - 1] = zero[q] ? 0ll : (long long)(fx_round_grid(b, E[q]) - C[q]);
        }
    }
}

// ---- integer stencil numerators (Eq. 13 points, sixth order) ---------------

// 45 (F1 - F-1) - 9 (F2 - F-2) + (F3 - F-3): first derivative x 60 dx.
template <int AX, class V>
__device__ __forceinline__ long long nd1(const V &F) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    const long long a1 = F(ox, oy, oz) - F(-ox, -oy, -oz);
    const long long a2 = F(2 * ox, 2 * oy, 2 * oz) - F(-2 * ox, -2 * oy, -2 * oz);
    const long long a3 = F(3 * ox, 3 * oy, 3 * oz) - F(-3 * ox, -3 * oy, -3 * oz);
    return 45 * a1 - 9 * a2 + a3;
}

// -490 F0 + 270 (F1 + F-1) - 27 (F2 + F-2) + 2 (F3 + F-3): second derivative x 180 dx^2.
template <int AX, class V>
__device__ __forceinline__ long long nd2(const V &F, long long F0) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    const long long s1 = F(ox, oy, oz) + F(-ox, -oy, -oz);
    const long long s2 = F(2 * ox, 2 * oy, 2 * oz) + F(-2 * ox, -2 * oy, -2 * oz);
    const long long s3 = F(3 * ox, 3 * oy, 3 * oz) + F(-3 * ox, -3 * oy, -3 * oz);
    return -490 * F0 + 270 * s1 - 27 * s2 + 2 * s3;
}

// 270 S1 - 27 S2 + 2 S3 over the face diagonals: mixed derivative x 720 dx^2.
template <int A, int B, class V>
__device__ __forceinline__ long long ndab(const V &F) {
    constexpr int ax = A == 0, ay = A == 1, az = A == 2;
    constexpr int bx = B == 0, by = B == 1, bz = B == 2;
    long long S[3];
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const long long pp = F(m * (ax + bx), m * (ay + by), m * (az + bz));
        const long long mm = F(-m * (ax + bx), -m * (ay + by), -m * (az + bz));
        const long long pm = F(m * (ax - bx), m * (ay - by), m * (az - bz));
        const long long mp = F(-m * (ax - bx), -m * (ay - by), -m * (az - bz));
        S[m - 1] = (pp + mm) - (pm + mp);
    }
    return 270 * S[0] - 27 * S[1] + 2 * S[2];
}

// (double)N 2^k exactly for the integer numerator N, by adding k to the
// exponent field of the converted value (k_hi = k << 20, the exponent's place in
// the high word); 0 stays 0.  Every product stays normal: 1 <= |N| < 2^63 and
// the plan keeps 2^(E - FX_BITS) within [2^-1010, 2^910].
__device__ __forceinline__ double fx_scaled(long long N, int k_hi) {
    const double v = (double)N;
    return N == 0 ? 0.0 : __hiloint2double(__double2hiint(v) + k_hi, __double2loint(v));
}

// Coefficients of the converted numerators (host side); the field scales
// 2^(E - FX_BITS) come from the device plan.  Every coefficient through which a
// term enters the right-hand side also carries the step dt (dts below; the host
// takes this path only for |dt| in [1e-100, 1e100], so that 1 / dt^2 stays in
// range).  The RHS so formed is dt times Eqs. B.1-B.4, and the RK update adds it
// to alpha w without multiplying it by dt.
struct FxCoefs {
    double c1dt;       // dts c1, c1 = 1 / (60 dx): first derivatives in the RHS and B = curl A
    double nu180;      // dts nu / (180 dx^2): nu lap u
    double nu2160;     // dts (nu + 3 zeta) / (2160 dx^2): (nu / 3 + zeta) grad(div u)
    double inv180dx2;  // 1 / (180 dx^2): lap A (in j, and times eta dts in Eq. B.4)
    double inv720dx2;  // 1 / (720 dx^2): grad(div A)
    double two_nu_c1sq;  // dts 2 nu c1^2: 2 nu S : S and 2 nu S grad ln rho from unscaled gradients
    double K_c1sq;       // dts K c1^2: K |grad xi|^2 (conduction)
    double zeta_c1sq;    // dts zeta c1^2: zeta (div u)^2
    double eta_dt;       // dts eta
    double hc_dt;        // dts (H - C)
    double K_dt;         // dts K
    double amp_dt[3];    // dts times the forcing amplitudes
    double inv_dt2;      // 1 / dts^2: |B|^2 of the CFL speed from the dts-scaled B
};

// Eqs. B.1-B.4 at one cell as cell_physics computes them, times dts (the step
// folded into the coefficients of FxCoefs), with the gradients of ln rho, s and
// u passed without the grid factor c1 = 1 / (60 dx) (the integer stencil
// numerators after their field scale): every term is linear or quadratic in
// them, so c1 enters the coefficients (dts c1 for the advection terms inside
// their fused multiply-adds, dts c1 cs^2 for the pressure term, dts c1^2 in
// 2 nu, K and zeta) instead of 15 multiplications per cell on the FP64 pipe.
// B = curl A comes scaled by dts c1 (it meets c1 in three places, and dts
// reaches the Lorentz force and the induction through it).
template <bool EXT>
__device__ __forceinline__ void cell_physics_fx(const double (&u)[3], const double (&GL)[3],
                                                const double (&GS)[3], const double (&GU)[3][3],
                                                const double (&B)[3], const double (&viscl)[3],
                                                const double (&lapa)[3], const double (&J)[3],
                                                const DevCoefs<double> &k, const FxCoefs &fc,
                                                const double frc[3], double out[NF], double *cfl,
                                                double lapxi, const Thermo<double> &th) {
    const double c1 = fc.c1dt;
    const double rho_inv = th.rho_inv, cs2 = th.cs2, inv_T = th.inv_T;
    const double divR = GU[0][0] + GU[1][1] + GU[2][2];  // div u / c1
    const double third_div = divR * (1.0 / 3.0);
    // traceless rate of strain S / c1
    const double Sxx = GU[0][0] - third_div, Syy = GU[1][1] - third_div, Szz = GU[2][2] - third_div;
    const double Sxy = 0.5 * (GU[0][1] + GU[1][0]);
    const double Sxz = 0.5 * (GU[0][2] + GU[2][0]);
    const double Syz = 0.5 * (GU[1][2] + GU[2][1]);
    const double SS2 = Sxx * Sxx + Syy * Syy + Szz * Szz + 2.0 * (Sxy * Sxy + Sxz * Sxz + Syz * Syz);
    const double SG[3] = {Sxx * GL[0] + Sxy * GL[1] + Sxz * GL[2],
                          Sxy * GL[0] + Syy * GL[1] + Syz * GL[2],
                          Sxz * GL[0] + Syz * GL[1] + Szz * GL[2]};
    const double JxB[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2],
                           J[0] * B[1] - J[1] * B[0]};
    const double UxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2],
                           u[0] * B[1] - u[1] * B[0]};
    const double J2 = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
    // Eq. B.1
    out[0] = -(c1 * (u[0] * GL[0] + u[1] * GL[1] + u[2] * GL[2] + divR));
    // Eq. B.2
    const double c1cs2 = c1 * cs2;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double adv = u[0] * GU[m][0] + u[1] * GU[m][1] + u[2] * GU[m][2];
        const double press = c1cs2 * (GS[m] * k.inv_cp + GL[m]);
        const double visc = viscl[m] + fc.two_nu_c1sq * SG[m];
        out[1 + m] = fma(-c1, adv, visc) - press + JxB[m] * rho_inv + frc[m];
    }
    // Eq. B.3
    out[4] = fma(-c1, u[0] * GS[0] + u[1] * GS[1] + u[2] * GS[2],
                 (fc.eta_dt * J2 * rho_inv + fc.two_nu_c1sq * SS2) * inv_T);
    if (EXT) {
        double gxi2 = 0.0;  // |grad xi|^2 / c1^2
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const double gxi = k.gamma_cp * GS[m] + k.gm1 * GL[m];
            gxi2 += gxi * gxi;
        }
        out[4] += (fc.hc_dt * rho_inv + fc.zeta_c1sq * divR * divR) * inv_T +
                  rho_inv * (fc.K_dt * lapxi + fc.K_c1sq * gxi2);
    }
    // Eq. B.4
#pragma unroll
    for (int m = 0; m < 3; ++m) out[5 + m] = UxB[m] + fc.eta_dt * lapa[m];
    if (cfl) {
        const double b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) * fc.inv_dt2;
        const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        *cfl = sqrt(u2) + sqrt(cs2 + b2 * rho_inv);
    }
}

// One (x, y) column of the integer-sum substep.  PF: per-field scales (FX_FIELD),
// so sums across the components of u or A are formed in binary64 from per-field
// integer numerators; otherwise one scale per group (FX_GROUP).
template <bool PF, bool CFL, bool EXT>
__device__ __forceinline__ void fx_column(const SubstepArgs<double, double> &a, const FxPtrs &fx,
                                          const FxCoefs &fc, const FxPlan *plan,
                                          const double *etab, int i, int j, double &cfl) {
    // Each field's scale 2^(E - FX_BITS) is applied to its converted numerators
    // by an exponent add on the integer pipe (fx_scaled), so only the grid
    // coefficients -- kernel parameters, read from the constant bank -- multiply
    // on the FP64 pipe, and no scaled coefficient occupies registers (the
    // kernels sit at 255 registers).  In FX_GROUP the components of u and of A
    // share their exponent.
    int kh[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) kh[q] = (plan->E[q] - FX_BITS) << 20;
    // first derivative of field q from its numerator; the gradients of ln rho, s
    // and u stay without the factor c1 (cell_physics_fx applies it)
    auto d1 = [&](long long N, int q) -> double { return fx_scaled(N, kh[q]) * fc.c1dt; };
    auto d1r = [&](long long N, int q) -> double { return fx_scaled(N, kh[q]); };
    const int k0 = blockIdx.z * a.zchunk;
    const int k1 = min(k0 + a.zchunk, a.g.nz);
    IdxPeriodic32 ix;
    ix.set_xy(i, j, a.g);
    double2 exy = make_double2(0.0, 0.0);
    if (a.force_on) {
        const double2 ex = a.ftab[i], ey = a.ftab[a.g.nx + j];
        exy.x = ex.x * ey.x - ex.y * ey.y;
        exy.y = ex.x * ey.y + ex.y * ey.x;
    }
    for (int kk = k0; kk < k1; ++kk) {
        ix.set_z(kk, a.g);
        const long long o = ix(0, 0, 0);
        // Centre values (the binary64 state) and the thermodynamic factors: at the
        // top of the cell in the CFL variant (substep 0), after the stencil sums in
        // the other; each placement measured fastest for its variant at 256^3
        // (8.30 against 8.78 ms, 7.89 against 8.64 ms), a matter of register
        // allocation at 255 registers.
        double lnrho = 0.0, ss = 0.0;
        Thermo<double> th;
        if constexpr (CFL) {
            lnrho = ldg(a.fin[0] + o);
            ss = ldg(a.fin[4] + o);
            th = thermo_factors<double>(lnrho, ss, a.k, etab);
        }
        double frc[3] = {0.0, 0.0, 0.0};
        if (a.force_on) {
            const double2 ez = a.ftab[a.g.nx + a.g.ny + kk];
            const double cph = exy.x * ez.x - exy.y * ez.y;
            frc[0] = fc.amp_dt[0] * cph;
            frc[1] = fc.amp_dt[1] * cph;
            frc[2] = fc.amp_dt[2] * cph;
        }
        const GlobalView<long long, IdxPeriodic32> Fl{fx.F[0], ix}, Fs{fx.F[4], ix};
        const GlobalView<long long, IdxPeriodic32> Fu[3] = {{fx.F[1], ix}, {fx.F[2], ix},
                                                             {fx.F[3], ix}};
        const GlobalView<long long, IdxPeriodic32> Fa[3] = {{fx.F[5], ix}, {fx.F[6], ix},
                                                             {fx.F[7], ix}};
        // first derivatives
        double gl[3], gs[3], gu[3][3], B[3];
        gl[0] = d1r(nd1<0>(Fl), 0);
        gl[1] = d1r(nd1<1>(Fl), 0);
        gl[2] = d1r(nd1<2>(Fl), 0);
        gs[0] = d1r(nd1<0>(Fs), 4);
        gs[1] = d1r(nd1<1>(Fs), 4);
        gs[2] = d1r(nd1<2>(Fs), 4);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int qu = PF ? 1 + m : 1;  // one live exponent in FX_GROUP
            gu[m][0] = d1r(nd1<0>(Fu[m]), qu);
            gu[m][1] = d1r(nd1<1>(Fu[m]), qu);
            gu[m][2] = d1r(nd1<2>(Fu[m]), qu);
        }
        if constexpr (PF) {
            B[0] = (fx_scaled(nd1<1>(Fa[2]), kh[7]) - fx_scaled(nd1<2>(Fa[1]), kh[6])) * fc.c1dt;
            B[1] = (fx_scaled(nd1<2>(Fa[0]), kh[5]) - fx_scaled(nd1<0>(Fa[2]), kh[7])) * fc.c1dt;
            B[2] = (fx_scaled(nd1<0>(Fa[1]), kh[6]) - fx_scaled(nd1<1>(Fa[0]), kh[5])) * fc.c1dt;
        } else {
            B[0] = d1(nd1<1>(Fa[2]) - nd1<2>(Fa[1]), 5);
            B[1] = d1(nd1<2>(Fa[0]) - nd1<0>(Fa[2]), 5);
            B[2] = d1(nd1<0>(Fa[1]) - nd1<1>(Fa[0]), 5);
        }
        // lap V_i = sum_a N2_aa(V_i) / (180 dx^2);
        // grad(div V)_i = [4 N2_ii(V_i) + NX_ij(V_j) + NX_ik(V_k)] / (720 dx^2);
        // component C of V contributes 4 N2_CC to entry C and its two mixed
        // numerators to the other two entries.
        double viscl[3], lapa[3], J[3];
        if constexpr (PF) {
            // per-field scaled numerators, summed across components in binary64
            double LU[3], GU[3], LA[3], GA[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int b1 = c == 0 ? 1 : 0, b2 = c == 2 ? 1 : 2;
                {
                    const long long c0 = Fu[c](0, 0, 0);
                    const long long xx = nd2<0>(Fu[c], c0), yy = nd2<1>(Fu[c], c0),
                                    zz = nd2<2>(Fu[c], c0);
                    const int k = kh[1 + c];
                    LU[c] = fx_scaled(xx + yy + zz, k);
                    const double own = fx_scaled(4 * (c == 0 ? xx : (c == 1 ? yy : zz)), k);
                    const double x1 = fx_scaled(c == 2 ? ndab<0, 2>(Fu[c]) : ndab<0, 1>(Fu[c]), k);
                    const double x2 = fx_scaled(c == 0 ? ndab<0, 2>(Fu[c]) : ndab<1, 2>(Fu[c]), k);
                    if (c == 0) {
                        GU[0] = own;
                        GU[1] = x1;
                        GU[2] = x2;
                    } else {
                        GU[c] += own;
                        GU[b1] += x1;
                        GU[b2] += x2;
                    }
                }
                {
                    const long long c0 = Fa[c](0, 0, 0);
                    const long long xx = nd2<0>(Fa[c], c0), yy = nd2<1>(Fa[c], c0),
                                    zz = nd2<2>(Fa[c], c0);
                    const int k = kh[5 + c];
                    LA[c] = fx_scaled(xx + yy + zz, k);
                    const double own = fx_scaled(4 * (c == 0 ? xx : (c == 1 ? yy : zz)), k);
                    const double x1 = fx_scaled(c == 2 ? ndab<0, 2>(Fa[c]) : ndab<0, 1>(Fa[c]), k);
                    const double x2 = fx_scaled(c == 0 ? ndab<0, 2>(Fa[c]) : ndab<1, 2>(Fa[c]), k);
                    if (c == 0) {
                        GA[0] = own;
                        GA[1] = x1;
                        GA[2] = x2;
                    } else {
                        GA[c] += own;
                        GA[b1] += x1;
                        GA[b2] += x2;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                viscl[m] = fma(LU[m], fc.nu180, GU[m] * fc.nu2160);
                lapa[m] = LA[m] * fc.inv180dx2;
                J[m] = fma(GA[m], fc.inv720dx2, -lapa[m]);
            }
        } else {
            long long LU[3], GU[3];
            {
                const long long c0 = Fu[0](0, 0, 0);
                const long long xx = nd2<0>(Fu[0], c0), yy = nd2<1>(Fu[0], c0), zz = nd2<2>(Fu[0], c0);
                LU[0] = xx + yy + zz;
                GU[0] = 4 * xx;
                GU[1] = ndab<0, 1>(Fu[0]);
                GU[2] = ndab<0, 2>(Fu[0]);
            }
            {
                const long long c0 = Fu[1](0, 0, 0);
                const long long xx = nd2<0>(Fu[1], c0), yy = nd2<1>(Fu[1], c0), zz = nd2<2>(Fu[1], c0);
                LU[1] = xx + yy + zz;
                GU[1] += 4 * yy;
                GU[0] += ndab<0, 1>(Fu[1]);
                GU[2] += ndab<1, 2>(Fu[1]);
            }
            {
                const long long c0 = Fu[2](0, 0, 0);
                const long long xx = nd2<0>(Fu[2], c0), yy = nd2<1>(Fu[2], c0), zz = nd2<2>(Fu[2], c0);
                LU[2] = xx + yy + zz;
                GU[2] += 4 * zz;
                GU[0] += ndab<0, 2>(Fu[2]);
                GU[1] += ndab<1, 2>(Fu[2]);
            }
            // the same two sums for A; j = grad(div A) - lap A
            long long LA[3], GA[3];
            {
                const long long c0 = Fa[0](0, 0, 0);
                const long long xx = nd2<0>(Fa[0], c0), yy = nd2<1>(Fa[0], c0), zz = nd2<2>(Fa[0], c0);
                LA[0] = xx + yy + zz;
                GA[0] = 4 * xx;
                GA[1] = ndab<0, 1>(Fa[0]);
                GA[2] = ndab<0, 2>(Fa[0]);
            }
            {
                const long long c0 = Fa[1](0, 0, 0);
                const long long xx = nd2<0>(Fa[1], c0), yy = nd2<1>(Fa[1], c0), zz = nd2<2>(Fa[1], c0);
                LA[1] = xx + yy + zz;
                GA[1] += 4 * yy;
                GA[0] += ndab<0, 1>(Fa[1]);
                GA[2] += ndab<1, 2>(Fa[1]);
            }
            {
                const long long c0 = Fa[2](0, 0, 0);
                const long long xx = nd2<0>(Fa[2], c0), yy = nd2<1>(Fa[2], c0), zz = nd2<2>(Fa[2], c0);
                LA[2] = xx + yy + zz;
                GA[2] += 4 * zz;
                GA[0] += ndab<0, 2>(Fa[2]);
                GA[1] += ndab<1, 2>(Fa[2]);
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                viscl[m] = fma(fx_scaled(LU[m], kh[1]), fc.nu180, fx_scaled(GU[m], kh[1]) * fc.nu2160);
                lapa[m] = fx_scaled(LA[m], kh[5]) * fc.inv180dx2;
                J[m] = fma(fx_scaled(GA[m], kh[5]), fc.inv720dx2, -lapa[m]);
            }
        }
        // EXT: lap xi = gamma / c_p lap s + (gamma - 1) lap ln rho (conduction)
        double lapxi = 0.0;
        if (EXT) {
            const long long l0 = Fl(0, 0, 0), s0 = Fs(0, 0, 0);
            const long long LL = nd2<0>(Fl, l0) + nd2<1>(Fl, l0) + nd2<2>(Fl, l0);
            const long long LS = nd2<0>(Fs, s0) + nd2<1>(Fs, s0) + nd2<2>(Fs, s0);
            lapxi = a.k.gamma_cp * (fx_scaled(LS, kh[4]) * fc.inv180dx2) +
                    a.k.gm1 * (fx_scaled(LL, kh[0]) * fc.inv180dx2);
        }
        if constexpr (!CFL) {
            lnrho = ldg(a.fin[0] + o);
            ss = ldg(a.fin[4] + o);
            th = thermo_factors<double>(lnrho, ss, a.k, etab);
        }
        const double u[3] = {ldg(a.fin[1] + o), ldg(a.fin[2] + o), ldg(a.fin[3] + o)};
        double rhs[NF];
        if (CFL) {
            double c;
            cell_physics_fx<EXT>(u, gl, gs, gu, B, viscl, lapa, J, a.k, fc, frc, rhs, &c, lapxi, th);
            cfl = (c > cfl || c != c) ? c : cfl;
        } else {
            cell_physics_fx<EXT>(u, gl, gs, gu, B, viscl, lapa, J, a.k, fc, frc, rhs, nullptr, lapxi,
                                 th);
        }
        // the RK update of rk_update, the RHS already multiplied by dt
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            double wn = rhs[q];
            if (!a.s0) wn = a.alpha * a.w[q][o] + wn;
            a.w[q][o] = wn;
            a.fout[q][o] = ldg(a.fin[q] + o) + a.beta * wn;
        }
    }
}

// The substep in one mode of the plan: each mode is its own kernel (its own
// register allocation: in one kernel with all three bodies ptxas spilled the
// group-scale body, 16 B per cell at 128^3, and it ran 3-10% slower), launched
// every substep; the two kernels whose mode the plan did not choose return at
// once.  Two CTAs of 128 threads per SM (8 warps, as many as 255 registers
// allow): with the minimum stated, ptxas keeps the body within 255 registers
// (a cap of 168 registers for 12 warps spills and is slower).
template <bool PF, bool CFL, bool EXT = false>
__global__ void __launch_bounds__(128, 2) substep_fx_kernel(const SubstepArgs<double, double> a,
                                                         const FxPtrs fx, FxCoefs fc,
                                                         const FxPlan *plan) {
    if (plan->mode != (PF ? FX_FIELD : FX_GROUP)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = i < a.g.nx && j < a.g.ny;
    __shared__ double etab[512];
    exp_tab_stage(etab);
    double cfl = 0.0;
    if (active) fx_column<PF, CFL, EXT>(a, fx, fc, plan, etab, i, j, cfl);
    if (CFL) block_max_to_global(cfl, a.cfl_max);
}

// FX_PLAIN: plain binary64 stencils, the arithmetic of AC_STENCIL_FP64.
template <bool CFL, bool EXT = false>
__global__ void __launch_bounds__(128) substep_fx_plain_kernel(const SubstepArgs<double, double> a,
                                                              const FxPlan *plan) {
    if (plan->mode != FX_PLAIN) return;
    substep_body<double, double, IdxPeriodic32, CFL, 3, EXT>(a);
}

}  // namespace ac
