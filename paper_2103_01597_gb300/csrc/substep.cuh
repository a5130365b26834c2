// Fused RHS + Runge-Kutta substep kernel (one pass over the grid), templated
// on the field type R, the accumulator type W, the addressing IX and the
// stencil radius RAD (order 2 RAD).
#pragma once

#include "stencil.cuh"

namespace ac {

template <typename R> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <typename R, typename W>
struct SubstepArgs {
    Geom g;
    const R *fin[NF];
    R *fout[NF];
    W *w[NF];
    DevCoefs<R> k;
    W alpha, beta, dt;
    int s0;      // substep 0: w is not read
    int zchunk;  // cells along z per thread
    int force_on;
    const typename Vec2<R>::type *ftab;  // e^{i theta_x}, e^{i theta_y}, e^{i (theta_z + phi)}
    R amp_e[3];
    unsigned long long *cfl_max;  // non-null at substep 0: max CFL speed of the input state
};

// Williamson 2N-storage update of one field at one cell:
// w <- alpha w + dt rhs (w not read when s0), f_out <- f_in + beta w.
template <typename R, typename W>
__device__ __forceinline__ void rk_update(const SubstepArgs<R, W> &a, int q, long long o, R rhs) {
    W wn = a.dt * (W)rhs;
    if (!a.s0) wn = a.alpha * a.w[q][o] + wn;
    a.w[q][o] = wn;
    a.fout[q][o] = (R)((W)ldg(a.fin[q] + o) + a.beta * wn);
}

// One (x, y) column: cells k0 .. k1-1.  With cfl_acc non-null the largest CFL
// speed of the input state is kept there.  `tx`, `ty`, `tz` are the forcing
// phase tables of the x, y and z axes (entries indexed by i, j, k).
template <typename R, typename W, class IX, int RAD = 3, bool EXT = false>
__device__ __forceinline__ void substep_column(const SubstepArgs<R, W> &a, int i, int j, int k0,
                                               int k1, const typename Vec2<R>::type *tx,
                                               const typename Vec2<R>::type *ty,
                                               const typename Vec2<R>::type *tz, R *cfl_acc) {
    using V2 = typename Vec2<R>::type;
    IX ix;
    ix.set_xy(i, j, a.g);
    // Forcing phase factor of this (x, y) column: e^{i (theta_x + theta_y)}.
    V2 exy = {(R)0, (R)0};
    if (a.force_on) {
        const V2 ex = tx[i], ey = ty[j];
        exy.x = ex.x * ey.x - ex.y * ey.y;
        exy.y = ex.x * ey.y + ex.y * ey.x;
    }
    for (int kk = k0; kk < k1; ++kk) {
        ix.set_z(kk, a.g);
        R frc[3] = {(R)0, (R)0, (R)0};
        if (a.force_on) {
            const V2 ez = tz[kk];
            const R cph = exy.x * ez.x - exy.y * ez.y;  // cos(k . x + phi)
            frc[0] = a.amp_e[0] * cph;
            frc[1] = a.amp_e[1] * cph;
            frc[2] = a.amp_e[2] * cph;
        }
        R rhs[NF];
        const GlobalCell<R, IX> cell{a.fin, ix};
        if (cfl_acc) {
            R c;
            cell_rhs<R, RAD, EXT>(cell, a.k, frc, rhs, &c);
            *cfl_acc = (c > *cfl_acc || c != c) ? c : *cfl_acc;
        } else {
            cell_rhs<R, RAD, EXT>(cell, a.k, frc, rhs);
        }
        const long long o = ix(0, 0, 0);
#pragma unroll
        for (int q = 0; q < NF; ++q) rk_update(a, q, o, rhs[q]);
    }
}

// CFL: also track the largest CFL speed of the input state (substep 0).
// EXT: the conduction, bulk-viscosity and heating/cooling terms of Eq. B.3.
template <typename R, typename W, class IX, bool CFL, int RAD, bool EXT>
__device__ __forceinline__ void substep_body(const SubstepArgs<R, W> &a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool active = i < a.g.nx && j < a.g.ny;
    const int k0 = blockIdx.z * a.zchunk;
    const int k1 = min(k0 + a.zchunk, a.g.nz);
    const auto *tx = a.ftab, *ty = a.ftab + a.g.nx, *tz = a.ftab + a.g.nx + a.g.ny;
    if (CFL) {
        R cfl = (R)0;
        if (active) substep_column<R, W, IX, RAD, EXT>(a, i, j, k0, k1, tx, ty, tz, &cfl);
        block_max_to_global((double)cfl, a.cfl_max);
    } else if (active) {
        substep_column<R, W, IX, RAD, EXT>(a, i, j, k0, k1, tx, ty, tz, nullptr);
    }
}

// A box [b0, b1) of the interior (x, y, z), for updates of one segment of a
// subdomain; blockIdx.z covers its z range in chunks of a.zchunk.  FLAT: the
// threads of 1-D blocks cover the box's x-y extent row by row, so a slab three
// cells thin still keeps every lane busy; otherwise 32 x 4 blocks tile it (whole
// warps on one row: the wider boxes' loads stay coalesced).  `ftab` holds the
// subdomain's own tables [nx | ny | nz].
struct Box {
    int b0[3], b1[3];
};

template <typename R, typename W, int RAD, bool EXT, bool FLAT>
__global__ void __launch_bounds__(128) substep_box_kernel(const SubstepArgs<R, W> a, Box box) {
    int i, j;
    if constexpr (FLAT) {
        const int ex = box.b1[0] - box.b0[0];
        const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (t >= (long long)ex * (box.b1[1] - box.b0[1])) return;
        i = box.b0[0] + (int)(t % ex);
        j = box.b0[1] + (int)(t / ex);
    } else {
        i = box.b0[0] + blockIdx.x * blockDim.x + threadIdx.x;
        j = box.b0[1] + blockIdx.y * blockDim.y + threadIdx.y;
        if (i >= box.b1[0] || j >= box.b1[1]) return;
    }
    const int k0 = box.b0[2] + blockIdx.z * a.zchunk;
    const int k1 = min(k0 + a.zchunk, box.b1[2]);
    const auto *tx = a.ftab, *ty = a.ftab + a.g.nx, *tz = a.ftab + a.g.nx + a.g.ny;
    substep_column<R, W, IdxPadded, RAD, EXT>(a, i, j, k0, k1, tx, ty, tz, nullptr);
}

template <typename R, typename W, class IX, bool CFL, int RAD = 3, bool EXT = false>
__global__ void __launch_bounds__(128) substep_kernel(const SubstepArgs<R, W> a) {
    substep_body<R, W, IX, CFL, RAD, EXT>(a);
}

// The same kernel with a stated minimum of two CTAs per SM, for binary32 at
// radius 4: ptxas then keeps more values in registers (255 instead of 130, 8
// instead of 12 warps per SM), measured 17% faster at 256^3.  At radius 1 and 2
// more registers cost more warps than they save.
template <typename R, typename W, class IX, bool CFL, int RAD, bool EXT>
__global__ void __launch_bounds__(128, 2) substep_kernel_2cta(const SubstepArgs<R, W> a) {
    substep_body<R, W, IX, CFL, RAD, EXT>(a);
}

template <typename R, typename W, class IX, bool CFL, int RAD, bool EXT>
void launch_substep_one(const SubstepArgs<R, W> &a, dim3 grid, dim3 block, cudaStream_t st) {
    if constexpr (sizeof(R) == 4 && RAD == 4)
        substep_kernel_2cta<R, W, IX, CFL, RAD, EXT><<<grid, block, 0, st>>>(a);
    else
        substep_kernel<R, W, IX, CFL, RAD, EXT><<<grid, block, 0, st>>>(a);
}

// Launch for radius RAD: periodic addressing with RAD-wide offsets, or the
// padded layout (halo 3, so RAD <= 3).
template <typename R, typename W, int RAD, bool EXT>
void launch_substep_r(const SubstepArgs<R, W> &a, bool padded, bool cfl, dim3 grid, dim3 block,
                      cudaStream_t st) {
    if (padded) {
        if constexpr (RAD <= 3) {
            if (cfl)
                launch_substep_one<R, W, IdxPadded, true, RAD, EXT>(a, grid, block, st);
            else
                launch_substep_one<R, W, IdxPadded, false, RAD, EXT>(a, grid, block, st);
        }
    } else if (a.g.elems < (1ll << 31) && !(sizeof(R) == 4 && RAD == 1)) {
        // 32-bit neighbour offsets (fewer registers).  Measured at 256^3: binary32
        // radius 2 and 4 gain 14% and 21% from them, radius 1 loses 17% (19.4
        // against 16.2 Gcell-updates/s) and keeps 64-bit ones; binary64 is unchanged.
        if (cfl)
            launch_substep_one<R, W, IdxPeriodicR<RAD, int>, true, RAD, EXT>(a, grid, block, st);
        else
            launch_substep_one<R, W, IdxPeriodicR<RAD, int>, false, RAD, EXT>(a, grid, block, st);
    } else {
        if (cfl)
            launch_substep_one<R, W, IdxPeriodicR<RAD>, true, RAD, EXT>(a, grid, block, st);
        else
            launch_substep_one<R, W, IdxPeriodicR<RAD>, false, RAD, EXT>(a, grid, block, st);
    }
}

template <typename R, typename W, int RAD>
void launch_substep_re(const SubstepArgs<R, W> &a, bool padded, bool cfl, bool ext, dim3 grid,
                       dim3 block, cudaStream_t st) {
    if (ext)
        launch_substep_r<R, W, RAD, true>(a, padded, cfl, grid, block, st);
    else
        launch_substep_r<R, W, RAD, false>(a, padded, cfl, grid, block, st);
}

template <typename R, typename W>
cudaError_t launch_substep_t(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    SubstepArgs<R, W> a;
    a.g = L.g;
    for (int q = 0; q < NF; ++q) {
        a.fin[q] = static_cast<const R *>(L.fin[q]);
        a.fout[q] = static_cast<R *>(L.fout[q]);
        a.w[q] = static_cast<W *>(L.w[q]);
    }
    a.k = to_dev<R>(L.c, L.ph);
    a.alpha = (W)L.alpha;
    a.beta = (W)L.beta;
    a.dt = (W)L.dt;
    a.s0 = L.s == 0;
    a.force_on = L.force.on;
    // The table block holds nx+ny+nz double2 entries followed by the same count of float2.
    const long long ntab = (long long)L.g.nx + L.g.ny + L.g.nz;
    if (sizeof(R) == 8)
        a.ftab = reinterpret_cast<const typename Vec2<R>::type *>(L.force.tab);
    else
        a.ftab = reinterpret_cast<const typename Vec2<R>::type *>(L.force.tab + ntab);
    for (int m = 0; m < 3; ++m) a.amp_e[m] = (R)L.force.amp_e[m];
    a.cfl_max = L.cfl_max;

    const dim3 block(32, 4, 1);
    const unsigned gx = (L.g.nx + block.x - 1) / block.x;
    const unsigned gy = (L.g.ny + block.y - 1) / block.y;
    // Enough z-slices for several waves of CTAs over 152 SMs, up to 16 cells per thread.
    const long long xy_blocks = (long long)gx * gy;
    int zchunk = (int)((xy_blocks * L.g.nz) / (8 * 152));
    zchunk = zchunk < 1 ? 1 : (zchunk > 16 ? 16 : zchunk);
    a.zchunk = zchunk;
    const dim3 grid(gx, gy, (L.g.nz + zchunk - 1) / zchunk);
    const bool cfl = a.cfl_max != nullptr;
    const bool ext = L.ph.ext();
    switch (L.c.radius) {
        case 1: launch_substep_re<R, W, 1>(a, L.g.padded, cfl, ext, grid, block, st); break;
        case 2: launch_substep_re<R, W, 2>(a, L.g.padded, cfl, ext, grid, block, st); break;
        case 4: launch_substep_re<R, W, 4>(a, L.g.padded, cfl, ext, grid, block, st); break;
        default: launch_substep_re<R, W, 3>(a, L.g.padded, cfl, ext, grid, block, st); break;
    }
    ++*launches;
    return cudaGetLastError();
}

}  // namespace ac
