// Binary64 substep with exact integer stencil sums (cubic periodic grids).
//
// GB300 executes two FP64 lanes per SM per cycle, so the binary64 substep is
// bound by its FP64 instruction count, most of which (about 400 of 600 per
// cell) are the additions and multiplications of the 54 stencils of Eq. 13.
// Here each field group (ln rho; u; s; A) is first written as int64 fixed
// point with one power-of-two scale per group, F = round(f 2^(50 - e)) with
// max |f| < 2^e, so |F| <= 2^50.  Every stencil numerator -- and every sum of
// numerators that share a coefficient (curl A, lap u, grad(div u), lap A,
// grad(div A)) -- is then an exact integer on the integer pipes (largest:
// 6744 |F| < 2^63), and only one int64 -> binary64 conversion and one
// multiplication per derivative term remain on the FP64 pipe.  The
// quantisation step, 2^-50 of the group's largest magnitude, is four binary64
// units in the last place at that magnitude; the centre values used by the
// physics and the Runge-Kutta update are the binary64 state itself.  The physics of Eqs. B.1-B.4 is unchanged
// binary64 code (cell_physics).
#pragma once

#include "substep.cuh"

namespace ac {

constexpr int FX_BITS = 50;

// Field -> group: 0 = ln rho, 1 = u, 2 = s, 3 = A.
__host__ __device__ __forceinline__ int fx_group(int q) {
    return q == 0 ? 0 : (q < 4 ? 1 : (q == 4 ? 2 : 3));
}

// Smallest e with m < 2^e for the binary64 m >= 0 held in `bits` (0 for m == 0,
// non-finite or subnormal m).
__device__ __forceinline__ int fx_exponent(unsigned long long bits) {
    const int eb = (int)((bits >> 52) & 0x7ff);
    if (eb == 0 || eb == 0x7ff) return 0;
    return eb - 1022;
}

// 2^k as a binary64 built from its bits (|k| < 1000).
__device__ __forceinline__ double fx_pow2(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// Largest |f| of each group over the current state (bits of binary64 values).
struct FxPtrs {
    const double *f[NF];
    long long *F[NF];
};

__global__ void fx_max_kernel(FxPtrs p, long long n, unsigned long long *gmax) {
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(p.f[q][t]) & 0x7fffffffffffffffull;
            const int gq = fx_group(q);
            m[gq] = b > m[gq] ? b : m[gq];
        }
    }
#pragma unroll
    for (int gq = 0; gq < 4; ++gq) {
        unsigned long long v = m[gq];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&gmax[gq], v);
    }
}

// F = round(f 2^(50 - e)) by integer operations on the binary64 bits (round
// half up in magnitude); values below the resolution become 0.
__global__ void fx_quantize_kernel(FxPtrs p, long long n, const unsigned long long *gmax) {
    int e[4];
#pragma unroll
    for (int gq = 0; gq < 4; ++gq) e[gq] = fx_exponent(gmax[gq]);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const long long b = __double_as_longlong(p.f[q][t]);
            const int eb = (int)((b >> 52) & 0x7ff);
            long long v = 0;
            if (eb != 0 && eb != 0x7ff) {
                const int sh = 1075 - FX_BITS + e[fx_group(q)] - eb;  // right shift of the significand
                if (sh > 0 && sh < 62) {
                    const long long mant = (b & 0xfffffffffffffll) | 0x10000000000000ll;
                    v = (mant + (1ll << (sh - 1))) >> sh;
                }
            }
            p.F[q][t] = b < 0 ? -v : v;
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

// Coefficients of the converted numerators; the group scales 2^(e - FX_BITS) are
// read from the max words on the device.
struct FxCoefs {
    double inv60dx;    // 1 / (60 dx): first derivatives
    double nu180;      // nu / (180 dx^2): nu lap u
    double nu2160;     // (nu + 3 zeta) / (2160 dx^2): (nu / 3 + zeta) grad(div u)
    double inv180dx2;  // 1 / (180 dx^2): lap A
    double inv720dx2;  // 1 / (720 dx^2): grad(div A)
};

// Two CTAs of 128 threads per SM (8 warps, as many as 255 registers allow): with
// the minimum stated, ptxas fits the kernel in 254 registers without the spills
// it otherwise makes (+4% at 256^3; a cap of 168 registers for 12 warps spills
// and is slower).
template <class IX, bool CFL, bool EXT = false>
__global__ void __launch_bounds__(128, 2) substep_fx_kernel(const SubstepArgs<double, double> a,
                                                         const FxPtrs fx, FxCoefs fc,
                                                         const unsigned long long *gmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = i < a.g.nx && j < a.g.ny;
    __shared__ double etab[512];
    exp_tab_stage(etab);
    double cfl = 0.0;
    if (active) {
        double sc[4];
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) sc[gq] = fx_pow2(fx_exponent(gmax[gq]) - FX_BITS);
        const double c1[4] = {sc[0] * fc.inv60dx, sc[1] * fc.inv60dx, sc[2] * fc.inv60dx,
                              sc[3] * fc.inv60dx};
        const double clu = sc[1] * fc.nu180;
        const double cgu = sc[1] * fc.nu2160;
        const double cla = sc[3] * fc.inv180dx2;
        const double cga = sc[3] * fc.inv720dx2;
        const int k0 = blockIdx.z * a.zchunk;
        const int k1 = min(k0 + a.zchunk, a.g.nz);
        IX ix;
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
                frc[0] = a.amp_e[0] * cph;
                frc[1] = a.amp_e[1] * cph;
                frc[2] = a.amp_e[2] * cph;
            }
            const GlobalView<long long, IX> Fl{fx.F[0], ix}, Fs{fx.F[4], ix};
            const GlobalView<long long, IX> Fu[3] = {{fx.F[1], ix}, {fx.F[2], ix}, {fx.F[3], ix}};
            const GlobalView<long long, IX> Fa[3] = {{fx.F[5], ix}, {fx.F[6], ix}, {fx.F[7], ix}};
            // first derivatives
            double gl[3], gs[3], gu[3][3], B[3];
            gl[0] = (double)nd1<0>(Fl) * c1[0];
            gl[1] = (double)nd1<1>(Fl) * c1[0];
            gl[2] = (double)nd1<2>(Fl) * c1[0];
            gs[0] = (double)nd1<0>(Fs) * c1[2];
            gs[1] = (double)nd1<1>(Fs) * c1[2];
            gs[2] = (double)nd1<2>(Fs) * c1[2];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                gu[m][0] = (double)nd1<0>(Fu[m]) * c1[1];
                gu[m][1] = (double)nd1<1>(Fu[m]) * c1[1];
                gu[m][2] = (double)nd1<2>(Fu[m]) * c1[1];
            }
            B[0] = (double)(nd1<1>(Fa[2]) - nd1<2>(Fa[1])) * c1[3];
            B[1] = (double)(nd1<2>(Fa[0]) - nd1<0>(Fa[2])) * c1[3];
            B[2] = (double)(nd1<0>(Fa[1]) - nd1<1>(Fa[0])) * c1[3];
            // lap u_i = sum_a N2_aa(u_i) / (180 dx^2);
            // grad(div u)_i = [4 N2_ii(u_i) + NX_ij(u_j) + NX_ik(u_k)] / (720 dx^2)
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
            double viscl[3], lapa[3], J[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                viscl[m] = (double)LU[m] * clu + (double)GU[m] * cgu;
                lapa[m] = (double)LA[m] * cla;
                J[m] = (double)GA[m] * cga - lapa[m];
            }
            // EXT: lap xi = gamma / c_p lap s + (gamma - 1) lap ln rho (conduction)
            double lapxi = 0.0;
            if (EXT) {
                const long long l0 = Fl(0, 0, 0), s0 = Fs(0, 0, 0);
                const long long LL = nd2<0>(Fl, l0) + nd2<1>(Fl, l0) + nd2<2>(Fl, l0);
                const long long LS = nd2<0>(Fs, s0) + nd2<1>(Fs, s0) + nd2<2>(Fs, s0);
                lapxi = a.k.gamma_cp * ((double)LS * (sc[2] * fc.inv180dx2)) +
                        a.k.gm1 * ((double)LL * (sc[0] * fc.inv180dx2));
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
                cell_physics<double, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, a.k, frc, rhs,
                                          &c, lapxi, th);
                cfl = (c > cfl || c != c) ? c : cfl;
            } else {
                cell_physics<double, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, a.k, frc, rhs,
                                          nullptr, lapxi, th);
            }
#pragma unroll
            for (int q = 0; q < NF; ++q) rk_update(a, q, o, rhs[q]);
        }
    }
    if (CFL) block_max_to_global(cfl, a.cfl_max);
}

}  // namespace ac
