// Shared-memory tiled, z-marching variant of the fused substep for binary32
// fields (periodic layout).
//
// Each CTA of 256 threads owns a TX x TY column tile (32 x 8 or 16 x 16) and
// walks a range of z.  A ring of shared-memory plane tiles holds, for all eight
// fields, the tile plus its radius-3 halo in x and y (x rounded out to 16-byte
// boundaries: columns x0-4 .. x0+TX+3); planes z-3 .. z+3 are resident while
// output plane z is computed and the next planes stream in with cp.async.
// Every stencil point of Eq. 13 is then one shared-memory load at a
// compile-time offset.  The periodic map of Sec. 3.3 is applied once per
// copied chunk.
#pragma once

#include "stencil_pair.cuh"
#include "substep.cuh"

namespace ac {

constexpr int TT_THREADS = 256;           // threads per CTA, launched as 32 x 8
constexpr int TT_PF = 2;                  // planes in flight beyond z+3 (at most; >= 1)
constexpr int TT_NP = 7 + TT_PF;          // ring slots
constexpr int TT_NW = TT_PF + 2;          // ring slots for the accumulator w of output planes

// Tile shape: TX x TY output cells, shared-memory rows of TX + 8 floats (x0-4 ..
// x0+TX+3) for rows y0-3 .. y0+TY+2.  Threads map to cells so that a warp's 32
// lanes read distinct banks at any common stencil offset: for TX = 32 a warp is
// one row; for TX = 16 its two half-warps lie two rows apart (2 x 24 floats =
// 16 banks), warp w holding rows r and r + 2, r = 4 (w / 2) + w % 2.
template <int TX_, int TY_>
struct TileShape {
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int ROW = TX + 8;        // floats per smem row
    static constexpr int ROWS = TY + 6;       // rows per field
    static constexpr int FIELD = ROW * ROWS;
    static constexpr int PLANE = NF * FIELD;  // floats per plane slot
    // copies per thread per plane: 16-byte chunks (x rounded to 16 B) or 4-byte elements
    static constexpr int VCH = NF * ROWS * (ROW / 4);
    static constexpr int VPT = (VCH + TT_THREADS - 1) / TT_THREADS;
    static constexpr int ECH = NF * ROWS * ROW;
    static constexpr int EPT = (ECH + TT_THREADS - 1) / TT_THREADS;
    static_assert(TX * TY == TT_THREADS && (TX == 32 || TX == 16), "tile shape");
    __device__ static __forceinline__ int tx(int tid) { return TX == 32 ? tid & 31 : tid & 15; }
    __device__ static __forceinline__ int ty(int tid) {
        if (TX == 32) return tid >> 5;
        const int w = tid >> 5;
        return 4 * (w >> 1) + (w & 1) + 2 * ((tid >> 4) & 1);
    }
};
using Tile32x8 = TileShape<32, 8>;
using Tile16x16 = TileShape<16, 16>;

// Linear thread index of a 32 x 8 launch.
__device__ __forceinline__ int tt_tid() { return threadIdx.y * 32 + threadIdx.x; }

template <typename W, class S>
constexpr size_t tt_smem_bytes() {
    return sizeof(float) * TT_NP * S::PLANE + sizeof(W) * TT_NW * NF * TT_THREADS;
}

// The values on the cell's own z-column (dx = dy = 0) come from a per-thread
// register queue of planes z-3 .. z+3; every other point from shared memory.
template <typename R, int ROW>
struct SmemView {
    const R *base;
    const int (&slot)[7];
    const R (&zq)[7];
    __device__ __forceinline__ R operator()(int dx, int dy, int dz) const {
        if (dx == 0 && dy == 0) return zq[dz + 3];
        return base[slot[dz + 3] + dy * ROW + dx];
    }
};

// Two fields with the same stencil points read together as a float2 (x: q1,
// y: q2) for the paired stencils of stencil_pair.cuh.
template <typename R, int ROW>
struct SmemPairView {
    const R *c1, *c2;
    const int (&slot)[7];
    const R (&z1)[7];
    const R (&z2)[7];
    __device__ __forceinline__ float2 operator()(int dx, int dy, int dz) const {
        if (dx == 0 && dy == 0) return make_float2(z1[dz + 3], z2[dz + 3]);
        const int o = slot[dz + 3] + dy * ROW + dx;
        return make_float2(c1[o], c2[o]);
    }
};

template <typename R, class S>
struct SmemCell {
    const R *cell;  // smem + (ty + 3) * S::ROW + tx + 4
    const int (&slot)[7];
    const R (&zq)[NF][7];
    __device__ __forceinline__ SmemView<R, S::ROW> operator[](int q) const {
        return {cell + q * S::FIELD, slot, zq[q]};
    }
    __device__ __forceinline__ SmemPairView<R, S::ROW> pair(int q1, int q2) const {
        return {cell + q1 * S::FIELD, cell + q2 * S::FIELD, slot, zq[q1], zq[q2]};
    }
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap_mod(int v, int n) {
    const int m = v % n;
    return m < 0 ? m + n : m;
}

// Per-thread copy list of one plane tile: for each copy, its shared-memory
// offset inside a ring slot and its source offset inside a z-plane (field base
// pointer folded in).  The periodic map of Sec. 3.3 is applied here once; only
// the z-plane offset changes from plane to plane.
template <class S, bool VEC>
struct TileCopies {
    static constexpr int N = VEC ? S::VPT : S::EPT;
    int soff[N];
    const float *src[N];
    int n;
    AC_BC_ONLY(long long bc_idx[N]; long long bc_lim;)
    template <class TA>
    __device__ __forceinline__ void init(const TA &ta, const Geom &g, int x0, int y0) {
        const int tid = tt_tid();
        n = 0;
        constexpr int CW = VEC ? 4 : 1;             // floats per copy
        constexpr int CH = S::ROW / CW;             // copies per row
        constexpr int TOTAL = NF * S::ROWS * CH;
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const int t = tid + u * TT_THREADS;
            if (t < TOTAL) {
                const int q = t / (S::ROWS * CH);
                const int rem = t - q * (S::ROWS * CH);
                const int r = rem / CH;
                const int c = rem - r * CH;
                const int gy = wrap_mod(y0 - 3 + r, g.ny);
                const int gx = wrap_mod(x0 - 4 + CW * c, g.nx);
                soff[u] = q * S::FIELD + r * S::ROW + CW * c;
                src[u] = ta.fin(q) + (long long)gy * g.px + gx;
                AC_BC_ONLY(bc_idx[u] = (long long)gy * g.px + gx; bc_lim = g.elems;)
                n = u + 1;
            }
        }
    }
    // Issue the copies of plane p (wrapped; p lies in [-3, nz + 2]) into `slot`.
    __device__ __forceinline__ void issue(float *slot, const Geom &g, int p) const {
        const int pw = g.nz >= 3 ? (p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p)) : wrap_mod(p, g.nz);
        const long long zoff = (long long)pw * g.pxy;
#pragma unroll
        for (int u = 0; u < N; ++u)
            if (u < n && AC_BC_RANGE(bc_idx[u] + zoff, VEC ? 4 : 1, bc_lim, AC_BC_TILE_IN)) {
                if (VEC)
                    cp_async16(slot + soff[u], src[u] + zoff);
                else
                    cp_async4(slot + soff[u], src[u] + zoff);
            }
    }
};

// Copy this thread's accumulator values of output plane z into a w ring slot.
template <typename W, class TA>
__device__ __forceinline__ void tile_load_w(W *wslot, const TA &ta, const Geom &g, int i, int j,
                                            int z, bool active) {
    if (!active) return;
    const int tid = tt_tid();
    const long long o = AC_BC((long long)z * g.pxy + (long long)j * g.px + i, g.elems, AC_BC_TILE_W);
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        if (sizeof(W) == 8) {
            cp_async8(wslot + q * TT_THREADS + tid, ta.w(q) + o);
        } else {
            cp_async4(wslot + q * TT_THREADS + tid, ta.w(q) + o);
        }
    }
}

// Argument adapter of the single-box launch: eight field pointers per buffer.
template <typename W>
struct TileOne {
    const SubstepArgs<float, W> &a;
    __device__ __forceinline__ const float *fin(int q) const { return a.fin[q]; }
    __device__ __forceinline__ float *fout(int q) const { return a.fout[q]; }
    __device__ __forceinline__ W *w(int q) const { return a.w[q]; }
    __device__ __forceinline__ const Geom &g() const { return a.g; }
    __device__ __forceinline__ const DevCoefs<float> &k() const { return a.k; }
    __device__ __forceinline__ W alpha() const { return a.alpha; }
    __device__ __forceinline__ W beta() const { return a.beta; }
    __device__ __forceinline__ W dt() const { return a.dt; }
    __device__ __forceinline__ int s0() const { return a.s0; }
    __device__ __forceinline__ int force_on() const { return a.force_on; }
    __device__ __forceinline__ const float2 *ftab() const { return a.ftab; }
    __device__ __forceinline__ float amp_e(int m) const { return a.amp_e[m]; }
    __device__ __forceinline__ unsigned long long *cfl_max() const { return a.cfl_max; }
};

// One output tile of shape S: columns [x0, x0+TX) x [y0, y0+TY), planes [z0,
// z1).  CFL: also fold the largest CFL speed of the input cells into
// ta.cfl_max().  The per-cell arithmetic does not depend on the shape.
template <class S, typename W, bool VEC, bool CFL, bool EXT, class TA>
__device__ __forceinline__ void tiled_body(const TA &ta, int x0, int y0, int z0, int z1,
                                           unsigned char *smem_raw) {
    constexpr int TT_PLANE = S::PLANE;
    float *sm = reinterpret_cast<float *>(smem_raw);
    W *wring = reinterpret_cast<W *>(sm + TT_NP * TT_PLANE);
    const Geom &g = ta.g();
    const int tid = tt_tid();
    const int tx = S::tx(tid), ty = S::ty(tid);
    const int i = x0 + tx, j = y0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const int force_on = ta.force_on();
    const int s0 = ta.s0();
    float cfl = 0.f;

    float2 exy = make_float2(0.f, 0.f);
    if (force_on && active) {
        const float2 ex = ta.ftab()[i], ey = ta.ftab()[g.nx + j];
        exy.x = ex.x * ey.x - ex.y * ey.y;
        exy.y = ex.x * ey.y + ex.y * ey.x;
    }
    TileCopies<S, VEC> cp;
    cp.init(ta, g, x0, y0);

    // One commit group per plane p, into ring offset `off`; it also carries w of
    // output plane p - 3 (w ring slot (p - 3 - z0) mod TT_NW).
    static_assert((TT_NW & (TT_NW - 1)) == 0, "w ring of a power-of-two size");
    auto issue = [&](int p, int off) {
        if (p <= z1 + 2) cp.issue(sm + off, g, p);
        const int zw = p - 3;
        if (!s0 && zw >= z0 && zw < z1)
            tile_load_w<W>(wring + ((zw - z0) & (TT_NW - 1)) * (NF * TT_THREADS), ta, g, i, j, zw,
                           active);
        cp_async_commit();
    };
    // planes z0-3 .. z0+2+TT_PF into slots 0 .. 5+TT_PF; each plane z's iteration, after
    // its barrier, issues plane z+3+TT_PF into the slot plane z-4 held (the slot
    // left free for z0)
    for (int p = z0 - 3; p <= z0 + 2 + TT_PF; ++p) issue(p, (p - z0 + 3) * TT_PLANE);
    int free_off = (6 + TT_PF) * TT_PLANE;

    float zq[NF][7];  // z-column of this thread's cell: planes z-3 .. z+3
    const float2 *ztab = force_on ? ta.ftab() + g.nx + g.ny : nullptr;
    float2 ez_next = force_on ? ztab[z0] : make_float2(0.f, 0.f);
    // ring offsets of planes z-3 .. z+3, rolled by one slot per plane
    int slot[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) slot[d] = d * TT_PLANE;
    for (int z = z0; z < z1; ++z) {
        const float2 ez = ez_next;  // forcing phase of plane z, loaded one plane ahead
        if (force_on && z + 1 < z1) ez_next = ztab[z + 1];
        cp_async_wait<TT_PF - 1>();  // plane z+3 (and w of plane z) have landed for this thread
        // ... and for every thread; every thread has also finished plane z-1, so
        // plane z-4's slot and the w slot of plane z-2 are free
        __syncthreads();
        issue(z + 3 + TT_PF, free_off);
        const float *ctr = sm + (ty + 3) * S::ROW + tx + 4;
        if (z == z0) {
#pragma unroll
            for (int q = 0; q < NF; ++q)
#pragma unroll
                for (int d = 0; d < 7; ++d) zq[q][d] = ctr[slot[d] + q * S::FIELD];
        } else {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
#pragma unroll
                for (int d = 0; d < 6; ++d) zq[q][d] = zq[q][d + 1];
                zq[q][6] = ctr[slot[6] + q * S::FIELD];
            }
        }
        if (active) {
            const SmemCell<float, S> cell{ctr, slot, zq};
            float frc[3] = {0.f, 0.f, 0.f};
            if (force_on) {
                const float cph = exy.x * ez.x - exy.y * ez.y;
                frc[0] = ta.amp_e(0) * cph;
                frc[1] = ta.amp_e(1) * cph;
                frc[2] = ta.amp_e(2) * cph;
            }
            float rhs[NF];
            // u_m with A_m and ln rho with s share every stencil: packed pairs
            if (CFL) {
                float c;
                cell_rhs_paired<EXT>(cell, ta.k(), frc, rhs, &c);
                cfl = (c > cfl || c != c) ? c : cfl;
            } else {
                cell_rhs_paired<EXT>(cell, ta.k(), frc, rhs, nullptr);
            }
            const long long o =
                AC_BC((long long)z * g.pxy + (long long)j * g.px + i, g.elems, AC_BC_TILE_OUT);
            const W *wz = wring + ((z - z0) & (TT_NW - 1)) * (NF * TT_THREADS) + tid;
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                W wn = ta.dt() * (W)rhs[q];
                if (!s0) wn = ta.alpha() * wz[q * TT_THREADS] + wn;
                ta.w(q)[o] = wn;
                ta.fout(q)[o] = (float)((W)zq[q][3] + ta.beta() * wn);
            }
        }
        free_off = slot[0];  // plane z-3's slot: refilled after the next barrier
#pragma unroll
        for (int d = 0; d < 6; ++d) slot[d] = slot[d + 1];
        slot[6] = slot[6] + TT_PLANE == TT_NP * TT_PLANE ? 0 : slot[6] + TT_PLANE;
    }
    cp_async_wait<0>();
    if (CFL) block_max_to_global((double)cfl, ta.cfl_max());
}

// Tile shape of the single-box launch.
using TileOneShape = Tile32x8;

template <typename W, bool VEC, bool CFL, bool EXT>
__global__ void __launch_bounds__(TT_THREADS, 1) substep_tiled_kernel(const SubstepArgs<float, W> a) {
    extern __shared__ __align__(128) unsigned char tt_smem_raw[];
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.g.nz);
    const TileOne<W> ta{a};
    tiled_body<TileOneShape, W, VEC, CFL, EXT>(ta, blockIdx.x * TileOneShape::TX,
                                               blockIdx.y * TileOneShape::TY, z0, z1, tt_smem_raw);
}

template <typename W, bool VEC, bool CFL, bool EXT>
static cudaError_t launch_tiled_variant_e(const SubstepArgs<float, W> &a, dim3 grid, dim3 block,
                                          cudaStream_t st) {
    const size_t smem = tt_smem_bytes<W, TileOneShape>();
    cudaError_t e = cudaFuncSetAttribute(substep_tiled_kernel<W, VEC, CFL, EXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    substep_tiled_kernel<W, VEC, CFL, EXT><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// EXT (the extra terms of Eq. B.3) is chosen from the coefficients.
template <typename W, bool VEC, bool CFL>
static cudaError_t launch_tiled_variant(const SubstepArgs<float, W> &a, dim3 grid, dim3 block,
                                        cudaStream_t st) {
    const bool ext = a.k.K != 0.f || a.k.zeta != 0.f || a.k.hc != 0.f;
    return ext ? launch_tiled_variant_e<W, VEC, CFL, true>(a, grid, block, st)
               : launch_tiled_variant_e<W, VEC, CFL, false>(a, grid, block, st);
}

// Launch the tiled kernel for binary32 fields in the periodic layout.
template <typename W>
cudaError_t launch_substep_tiled_t(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    SubstepArgs<float, W> a;
    a.g = L.g;
    for (int q = 0; q < NF; ++q) {
        a.fin[q] = static_cast<const float *>(L.fin[q]);
        a.fout[q] = static_cast<float *>(L.fout[q]);
        a.w[q] = static_cast<W *>(L.w[q]);
    }
    a.k = to_dev<float>(L.c, L.ph);
    a.alpha = (W)L.alpha;
    a.beta = (W)L.beta;
    a.dt = (W)L.dt;
    a.s0 = L.s == 0;
    a.force_on = L.force.on;
    const long long ntab = (long long)L.g.nx + L.g.ny + L.g.nz;
    a.ftab = reinterpret_cast<const float2 *>(L.force.tab + ntab);
    for (int m = 0; m < 3; ++m) a.amp_e[m] = (float)L.force.amp_e[m];
    a.cfl_max = L.cfl_max;

    const unsigned gx = (L.g.nx + TileOneShape::TX - 1) / TileOneShape::TX;
    const unsigned gy = (L.g.ny + TileOneShape::TY - 1) / TileOneShape::TY;
    // z range per CTA: up to 128 planes, fewer until there are at least two CTAs per SM.
    int zc = L.g.nz < 128 ? L.g.nz : 128;
    while (zc > 16 && (long long)gx * gy * ((L.g.nz + zc - 1) / zc) < 2 * 152) zc = (zc + 1) / 2;
    a.zchunk = zc;
    const dim3 grid(gx, gy, (L.g.nz + zc - 1) / zc);
    const dim3 block(32, 8, 1);
    const bool vec = (L.g.nx % 4) == 0;
    const bool cfl = a.cfl_max != nullptr;
    cudaError_t e;
    if (vec)
        e = cfl ? launch_tiled_variant<W, true, true>(a, grid, block, st)
                : launch_tiled_variant<W, true, false>(a, grid, block, st);
    else
        e = cfl ? launch_tiled_variant<W, false, true>(a, grid, block, st)
                : launch_tiled_variant<W, false, false>(a, grid, block, st);
    if (e != cudaSuccess) return e;
    ++*launches;
    return cudaGetLastError();
}

}  // namespace ac
