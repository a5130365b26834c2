// Paired binary32 stencils for the shared-memory tiled substep: the fields of
// Table B.1 come in pairs that share every stencil point and weight of Eq. 13
// -- (u_m, A_m) for m = x, y, z take first, second and mixed derivatives on
// the same points, (ln rho, s) first derivatives (and second ones for the
// conduction term) -- so each pair is evaluated by the packed binary32
// instructions of sm_100+ (FADD2, FMUL2, FFMA2 on a register pair), one
// instruction for both fields.  Every component is rounded as its scalar
// operation would be, in the same order as op_d1/op_d2/op_dab, so a field's
// derivatives equal the scalar path's bit for bit.
#pragma once

#include "stencil.cuh"

namespace ac {

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_bc(float c) { return make_float2(c, c); }

// First derivative of a pair along AX: sum_m c[m-1] (f_m - f_-m).
template <int AX, class PV>
__device__ __forceinline__ float2 p_d1(const PV &f, const float (&c)[MAX_RADIUS]) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    float2 sum = p_mul(p_bc(c[0]), p_sub(f(ox, oy, oz), f(-ox, -oy, -oz)));
#pragma unroll
    for (int m = 2; m <= 3; ++m)
        sum = p_fma(p_bc(c[m - 1]), p_sub(f(m * ox, m * oy, m * oz), f(-m * ox, -m * oy, -m * oz)),
                    sum);
    return sum;
}

// Second derivative of a pair along AX: c[0] f_0 + sum_m c[m] (f_m + f_-m).
template <int AX, class PV>
__device__ __forceinline__ float2 p_d2(const PV &f, float2 f0, const float (&c)[MAX_RADIUS + 1]) {
    constexpr int ox = AX == 0, oy = AX == 1, oz = AX == 2;
    float2 sum = p_mul(p_bc(c[0]), f0);
#pragma unroll
    for (int m = 1; m <= 3; ++m)
        sum = p_fma(p_bc(c[m]), p_add(f(m * ox, m * oy, m * oz), f(-m * ox, -m * oy, -m * oz)), sum);
    return sum;
}

// Mixed derivative of a pair in the plane of axes A < B from the face diagonals:
// sum_m c[m-1] S_m, S_m = (f(+m,+m) + f(-m,-m)) - (f(+m,-m) + f(-m,+m)).
template <int A, int B, class PV>
__device__ __forceinline__ float2 p_dab(const PV &f, const float (&c)[MAX_RADIUS]) {
    constexpr int ax = A == 0, ay = A == 1, az = A == 2;
    constexpr int bx = B == 0, by = B == 1, bz = B == 2;
    float2 S[3];
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
        const float2 pp = f(m * (ax + bx), m * (ay + by), m * (az + bz));
        const float2 mm = f(-m * (ax + bx), -m * (ay + by), -m * (az + bz));
        const float2 pm = f(m * (ax - bx), m * (ay - by), m * (az - bz));
        const float2 mp = f(-m * (ax - bx), -m * (ay - by), -m * (az - bz));
        S[m - 1] = p_sub(p_add(pp, mm), p_add(pm, mp));
    }
    float2 sum = p_mul(p_bc(c[0]), S[0]);
#pragma unroll
    for (int m = 2; m <= 3; ++m) sum = p_fma(p_bc(c[m - 1]), S[m - 1], sum);
    return sum;
}

// The second derivatives of one vector component pair V_C (u_C, A_C): the
// Laplacian, d_CC V_C and the two mixed derivatives d_C d_b V_C (b != C), as in
// component_second.
template <int C, class PV>
__device__ __forceinline__ void p_component_second(const PV &f, float2 f0, const DevCoefs<float> &k,
                                                   float2 &lap, float2 &dcc, float2 &cross_b1,
                                                   float2 &cross_b2) {
    const float2 dxx = p_d2<0>(f, f0, k.d2[0]);
    const float2 dyy = p_d2<1>(f, f0, k.d2[1]);
    const float2 dzz = p_d2<2>(f, f0, k.d2[2]);
    lap = p_add(p_add(dxx, dyy), dzz);
    constexpr int B1 = C == 0 ? 1 : 0;
    constexpr int B2 = C == 2 ? 1 : 2;
    dcc = C == 0 ? dxx : (C == 1 ? dyy : dzz);
    cross_b1 = p_dab<(C < B1 ? C : B1), (C < B1 ? B1 : C)>(f, k.dc[Plane<C, B1>::id]);
    cross_b2 = p_dab<(C < B2 ? C : B2), (C < B2 ? B2 : C)>(f, k.dc[Plane<C, B2>::id]);
}

// Eqs. B.1-B.4 at one cell from paired stencils.  `pair(q1, q2)` returns the
// view of fields q1 and q2 around the cell, as float2 values (x: q1, y: q2).
// The same terms, combinations and physics as cell_rhs<float, 3, EXT>.
template <bool EXT, class CELL2>
__device__ __forceinline__ void cell_rhs_paired(const CELL2 &f, const DevCoefs<float> &k,
                                                const float frc[3], float out[NF], float *cfl) {
    const auto ls = f.pair(0, 4);                                       // (ln rho, s)
    const auto ua0 = f.pair(1, 5), ua1 = f.pair(2, 6), ua2 = f.pair(3, 7);  // (u_m, A_m)
    const float2 c_ls = ls(0, 0, 0);
    const float2 c_ua[3] = {ua0(0, 0, 0), ua1(0, 0, 0), ua2(0, 0, 0)};
    const float lnrho = c_ls.x, ss = c_ls.y;
    const float u[3] = {c_ua[0].x, c_ua[1].x, c_ua[2].x};

    // first derivatives
    const float2 g_ls[3] = {p_d1<0>(ls, k.d1[0]), p_d1<1>(ls, k.d1[1]), p_d1<2>(ls, k.d1[2])};
    float2 g_ua[3][3];
    g_ua[0][0] = p_d1<0>(ua0, k.d1[0]);
    g_ua[0][1] = p_d1<1>(ua0, k.d1[1]);
    g_ua[0][2] = p_d1<2>(ua0, k.d1[2]);
    g_ua[1][0] = p_d1<0>(ua1, k.d1[0]);
    g_ua[1][1] = p_d1<1>(ua1, k.d1[1]);
    g_ua[1][2] = p_d1<2>(ua1, k.d1[2]);
    g_ua[2][0] = p_d1<0>(ua2, k.d1[0]);
    g_ua[2][1] = p_d1<1>(ua2, k.d1[1]);
    g_ua[2][2] = p_d1<2>(ua2, k.d1[2]);

    // second derivatives: Laplacians and grad(div .) of u and A together
    float2 lap[3], gd[3];
    {
        float2 dcc, c1, c2;
        p_component_second<0>(ua0, c_ua[0], k, lap[0], dcc, c1, c2);  // c1 = d_xy, c2 = d_xz
        gd[0] = dcc;
        gd[1] = c1;
        gd[2] = c2;
        p_component_second<1>(ua1, c_ua[1], k, lap[1], dcc, c1, c2);  // c1 = d_xy, c2 = d_yz
        gd[0] = p_add(gd[0], c1);
        gd[1] = p_add(gd[1], dcc);
        gd[2] = p_add(gd[2], c2);
        p_component_second<2>(ua2, c_ua[2], k, lap[2], dcc, c1, c2);  // c1 = d_xz, c2 = d_yz
        gd[0] = p_add(gd[0], c1);
        gd[1] = p_add(gd[1], c2);
        gd[2] = p_add(gd[2], dcc);
    }
    float gl[3], gs[3], gu[3][3], ga[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gl[a] = g_ls[a].x;
        gs[a] = g_ls[a].y;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            gu[m][a] = g_ua[m][a].x;
            ga[m][a] = g_ua[m][a].y;
        }
    }
    // B = curl A, j = grad(div A) - lap A, nu (lap u) + (nu / 3 + zeta) grad(div u)
    const float B[3] = {ga[2][1] - ga[1][2], ga[0][2] - ga[2][0], ga[1][0] - ga[0][1]};
    const float lapa[3] = {lap[0].y, lap[1].y, lap[2].y};
    const float J[3] = {gd[0].y - lap[0].y, gd[1].y - lap[1].y, gd[2].y - lap[2].y};
    float viscl[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) viscl[m] = k.nu * lap[m].x + k.nu3 * gd[m].x;
    float lapxi = 0.f;
    if (EXT) {  // lap xi = gamma / c_p lap s + (gamma - 1) lap ln rho
        const float2 l = p_add(p_add(p_d2<0>(ls, c_ls, k.d2[0]), p_d2<1>(ls, c_ls, k.d2[1])),
                               p_d2<2>(ls, c_ls, k.d2[2]));
        lapxi = k.gamma_cp * l.y + k.gm1 * l.x;
    }
    cell_physics<float, EXT>(lnrho, u, ss, gl, gs, gu, B, viscl, lapa, J, k, frc, out, cfl, lapxi,
                             thermo_factors<float>(lnrho, ss, k, nullptr));
}

}  // namespace ac
