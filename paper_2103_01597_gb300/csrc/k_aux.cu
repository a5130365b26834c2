// Auxiliary kernels: periodic halo fill (Sec. 3.3), forcing phase tables,
// host-format staging (load/store with precision conversion), and binary64
// reductions of fields and derived quantities.
#include <math.h>

#include "reduce.cuh"

namespace ac {

// ---------------------------------------------------------------------------
// Coefficients (host).  Central weights of order 2r on the points of Eq. 13
// (axes and face diagonals out to radius r), as integer numerators over a
// common denominator:
//   r = 3 (Sec. 4): d/dx (45, -9, 1) / 60 on (f_m - f_-m); d2/dx2 -49/18 on f_0
//          and (3/2, -3/20, 1/90) on (f_m + f_-m); d2/dxdy (270, -27, 2) / 720
//          on the diagonal sums S_m;
//   r = 1: (1) / 2;   -2, (1);                       (1) / 4;
//   r = 2: (8, -1) / 12;   -30/12, (16, -1) / 12;    (16, -1) / 48;
//   r = 4: (672, -168, 32, -3) / 840;   -14350/5040, (8064, -1008, 128, -9) / 5040;
//          (8064, -1008, 128, -9) / 20160.
// The mixed weights are the second-difference weights over 4 (S_m expands like
// 4 m^2 dx_a dx_b d_a d_b plus the same higher moments).
// ---------------------------------------------------------------------------
StencilCoefs make_coefs(const double dx[3], int radius) {
    StencilCoefs c = {};
    c.radius = radius;
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    if (radius == 3) {
        const double w1[3] = {45.0, -9.0, 1.0};
        const double w2[3] = {1.5, -0.15, 1.0 / 90.0};
        const double wc[3] = {270.0, -27.0, 2.0};
        for (int a = 0; a < 3; ++a) {
            for (int m = 0; m < 3; ++m) c.d1[a][m] = w1[m] / (60.0 * dx[a]);
            c.d2[a][0] = (-49.0 / 18.0) / (dx[a] * dx[a]);
            for (int m = 0; m < 3; ++m) c.d2[a][m + 1] = w2[m] / (dx[a] * dx[a]);
        }
        for (int pl = 0; pl < 3; ++pl)
            for (int m = 0; m < 3; ++m) c.dc[pl][m] = wc[m] / (720.0 * dx[pa[pl]] * dx[pb[pl]]);
        return c;
    }
    static const double n1[5][4] = {{0}, {1}, {8, -1}, {0}, {672, -168, 32, -3}};
    static const double q1[5] = {0, 2, 12, 0, 840};
    static const double n2[5][5] = {{0}, {-2, 1}, {-30, 16, -1}, {0}, {-14350, 8064, -1008, 128, -9}};
    static const double q2[5] = {0, 1, 12, 0, 5040};
    for (int a = 0; a < 3; ++a) {
        for (int m = 0; m < radius; ++m) c.d1[a][m] = n1[radius][m] / (q1[radius] * dx[a]);
        for (int m = 0; m <= radius; ++m) c.d2[a][m] = n2[radius][m] / (q2[radius] * dx[a] * dx[a]);
    }
    for (int pl = 0; pl < 3; ++pl)
        for (int m = 0; m < radius; ++m)
            c.dc[pl][m] = n2[radius][m + 1] / (4.0 * q2[radius] * dx[pa[pl]] * dx[pb[pl]]);
    return c;
}

PhysConsts make_phys(const ac_params &p) {
    PhysConsts c;
    c.nu = p.nu;
    c.eta = p.eta;
    c.inv_cp = 1.0 / p.cp;
    c.cs2_ref = p.cs0 * p.cs0 * exp(-(p.gamma - 1.0) * p.lnrho0);
    c.gamma_cp = p.gamma / p.cp;
    c.gm1 = p.gamma - 1.0;
    c.cp_gm1 = p.cp * (p.gamma - 1.0);
    c.K = 0.0;
    c.zeta = 0.0;
    c.hc = 0.0;
    return c;
}

// ---------------------------------------------------------------------------
// Periodic halo of the padded layout: every halo cell takes the value of its
// image ((s - r) mod n) + r per axis.  Halo cells are enumerated as three
// disjoint groups: the z-slabs (full padded planes), the y-slabs of the
// interior z range, and the x-slabs of the interior y and z ranges.
// ---------------------------------------------------------------------------

template <typename T>
__global__ void halo_kernel_pack(PtrPack<T> pk, Geom g, long long nz_slab, long long ny_slab,
                                 long long total) {
    T *arr = pk.p[blockIdx.y];
    const int mx = g.px;
    const int my = (int)(g.pxy / g.px);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (t < nz_slab) {
            const long long plane = (long long)mx * my;
            const long long zs = t / plane;
            const long long rem = t - zs * plane;
            k = zs < R ? (int)zs : (int)(g.nz + zs);
            j = (int)(rem / mx);
            i = (int)(rem - (long long)j * mx);
        } else if (t < nz_slab + ny_slab) {
            const long long u = t - nz_slab;
            const long long row = (long long)mx * 2 * R;
            const long long kz = u / row;
            const long long rem = u - kz * row;
            const int ys = (int)(rem / mx);
            k = (int)kz + R;
            j = ys < R ? ys : g.ny + ys;
            i = (int)(rem - (long long)ys * mx);
        } else {
            const long long u = t - nz_slab - ny_slab;
            const long long kz = u / ((long long)g.ny * 2 * R);
            const long long rem = u - kz * ((long long)g.ny * 2 * R);
            const int jy = (int)(rem / (2 * R));
            const int xs = (int)(rem - (long long)jy * 2 * R);
            k = (int)kz + R;
            j = jy + R;
            i = xs < R ? xs : g.nx + xs;
        }
        const int si = wrap_near(i - R, g.nx) + R;
        const int sj = wrap_near(j - R, g.ny) + R;
        const int sk = wrap_near(k - R, g.nz) + R;
        arr[(long long)k * g.pxy + (long long)j * mx + i] =
            arr[(long long)sk * g.pxy + (long long)sj * mx + si];
    }
}

cudaError_t launch_halo(int precision, const Geom &g, void *const f[NF], cudaStream_t st) {
    if (!g.padded) return cudaSuccess;
    const long long mx = g.px, my = g.pxy / g.px;
    const long long nz_slab = 2LL * R * mx * my;
    const long long ny_slab = (long long)g.nz * 2 * R * mx;
    const long long nx_slab = (long long)g.nz * g.ny * 2 * R;
    const long long total = nz_slab + ny_slab + nx_slab;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const dim3 grid((unsigned)blocks, NF);
    if (precision == AC_FP64) {
        PtrPack<double> pk;
        for (int q = 0; q < NF; ++q) pk.p[q] = static_cast<double *>(f[q]);
        halo_kernel_pack<double><<<grid, 256, 0, st>>>(pk, g, nz_slab, ny_slab, total);
    } else {
        PtrPack<float> pk;
        for (int q = 0; q < NF; ++q) pk.p[q] = static_cast<float *>(f[q]);
        halo_kernel_pack<float><<<grid, 256, 0, st>>>(pk, g, nz_slab, ny_slab, total);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Forcing tables: e^{i 2 pi k_a i / n_a} per axis (binary64, then a binary32
// copy), with the phase phi folded into the z table.  Layout: [nx | ny | nz]
// double2 entries, followed by the same count of float2 entries.
// ---------------------------------------------------------------------------
__global__ void forcing_table_kernel(int nx, int ny, int nz, int kx, int ky, int kz,
                                     double cphi, double sphi, double2 *tab) {
    const int total = nx + ny + nz;
    float2 *tabf = reinterpret_cast<float2 *>(tab + total);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int n, kk, i;
        if (t < nx) {
            n = nx; kk = kx; i = t;
        } else if (t < nx + ny) {
            n = ny; kk = ky; i = t - nx;
        } else {
            n = nz; kk = kz; i = t - nx - ny;
        }
        long long m = ((long long)kk * i) % n;
        if (m < 0) m += n;
        double s, c;
        sincospi(2.0 * (double)m / (double)n, &s, &c);
        if (t >= nx + ny) {  // rotate by phi
            const double c2 = c * cphi - s * sphi;
            const double s2 = s * cphi + c * sphi;
            c = c2;
            s = s2;
        }
        tab[t] = make_double2(c, s);
        tabf[t] = make_float2((float)c, (float)s);
    }
}

cudaError_t launch_forcing_table(const Geom &g, const int k[3], double phi, double2 *tab,
                                 cudaStream_t st) {
    const int total = g.nx + g.ny + g.nz;
    const int blocks = (total + 255) / 256;
    forcing_table_kernel<<<blocks, 256, 0, st>>>(g.nx, g.ny, g.nz, k[0], k[1], k[2], cos(phi),
                                                 sin(phi), tab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Staging: an unpadded float64 slab of nzc z-planes starting at z0 <-> a
// device array in its layout and precision.
// ---------------------------------------------------------------------------
// Host-format staging (S: binary64 or binary32, unpadded planes z0 .. z0 + nzc)
// to and from a device array of element type T in the handle's layout.
template <typename S, typename T>
__global__ void scatter_kernel(const S *__restrict__ stage, T *__restrict__ dst, Geom g, int z0,
                               long long count) {
    const long long plane = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long kz = t / plane;
        const long long rem = t - kz * plane;
        const long long j = rem / g.nx;
        const long long i = rem - j * g.nx;
        dst[g.origin + (z0 + kz) * g.pxy + j * g.px + i] = (T)stage[t];
    }
}

template <typename T, typename S>
__global__ void gather_kernel(const T *__restrict__ src, Geom g, int z0, long long count,
                              S *__restrict__ stage) {
    const long long plane = (long long)g.nx * g.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long kz = t / plane;
        const long long rem = t - kz * plane;
        const long long j = rem / g.nx;
        const long long i = rem - j * g.nx;
        stage[t] = (S)src[g.origin + (z0 + kz) * g.pxy + j * g.px + i];
    }
}

static unsigned grid_for(long long count) {
    long long b = (count + 255) / 256;
    return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <typename S>
static cudaError_t scatter_t(const S *stage, void *dst, int elem_size, const Geom &g, int z0,
                             int nzc, cudaStream_t st) {
    const long long count = (long long)g.nx * g.ny * nzc;
    if (elem_size == 8)
        scatter_kernel<S, double><<<grid_for(count), 256, 0, st>>>(stage, (double *)dst, g, z0, count);
    else
        scatter_kernel<S, float><<<grid_for(count), 256, 0, st>>>(stage, (float *)dst, g, z0, count);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t gather_t(const void *src, int elem_size, const Geom &g, int z0, int nzc,
                            S *stage, cudaStream_t st) {
    const long long count = (long long)g.nx * g.ny * nzc;
    if (elem_size == 8)
        gather_kernel<double, S><<<grid_for(count), 256, 0, st>>>((const double *)src, g, z0, count,
                                                                 stage);
    else
        gather_kernel<float, S><<<grid_for(count), 256, 0, st>>>((const float *)src, g, z0, count,
                                                                stage);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const double *stage, void *dst, int elem_size, const Geom &g, int z0,
                           int nzc, cudaStream_t st) {
    return scatter_t(stage, dst, elem_size, g, z0, nzc, st);
}
cudaError_t launch_gather(const void *src, int elem_size, const Geom &g, int z0, int nzc,
                          double *stage, cudaStream_t st) {
    return gather_t(src, elem_size, g, z0, nzc, stage, st);
}
cudaError_t launch_scatter_f32(const float *stage, void *dst, int elem_size, const Geom &g, int z0,
                               int nzc, cudaStream_t st) {
    return scatter_t(stage, dst, elem_size, g, z0, nzc, st);
}
cudaError_t launch_gather_f32(const void *src, int elem_size, const Geom &g, int z0, int nzc,
                              float *stage, cudaStream_t st) {
    return gather_t(src, elem_size, g, z0, nzc, stage, st);
}

// ---------------------------------------------------------------------------
// Reductions in binary64.  Pass 1: each block reduces a grid-stride share of
// the cells into partials[block] and flags[block] (non-finite seen); pass 2:
// one block reduces the partials in a fixed order, so results are
// deterministic for a given grid.
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 8 * 152;  // eight 256-thread CTAs per SM

int reduce_max_blocks() { return RED_MAX_BLOCKS; }

// Rows of constant (y, z) are dealt to warps; lanes walk x.  The periodic
// offsets of y and z are set once per row, those of x once per cell.
template <typename R, class IX, int RAD = 3>
__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(PtrPack<const R> pk, Geom g,
                                                             DevCoefs<R> k, int op, int quantity,
                                                             double *partials,
                                                             unsigned int *flags) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long rows = (long long)g.ny * g.nz;
    double acc = red_init(op);
    unsigned int bad = 0;
    for (long long row = (long long)blockIdx.x * (RED_THREADS / 32) + wid; row < rows;
         row += (long long)gridDim.x * (RED_THREADS / 32)) {
        const int kz = (int)(row / g.ny);
        const int j = (int)(row - (long long)kz * g.ny);
        IX ix;
        ix.set_xy(0, j, g);
        ix.set_z(kz, g);
        for (int i = lane; i < g.nx; i += 32) {
            ix.set_x(i, g);
            const double v = cell_quantity<R, IX, RAD>(pk.p, ix, k, quantity);
            if (!isfinite(v)) bad = 1;
            acc = red_combine(op, acc, op == AC_RMS ? v * v : v);
        }
    }
    __shared__ double sh[RED_THREADS / 32];
    __shared__ unsigned int shb[RED_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc = red_combine(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        sh[wid] = acc;
        shb[wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        unsigned int b = shb[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) {
            r = red_combine(op, r, sh[w]);
            b |= shb[w];
        }
        partials[blockIdx.x] = r;
        flags[blockIdx.x] = b;
    }
}

__global__ void reduce_final_kernel(const double *partials, const unsigned int *flags, int n,
                                    int op, double count, double *result) {
    __shared__ double sh[RED_THREADS];
    __shared__ unsigned int shb[RED_THREADS];
    double acc = red_init(op);
    unsigned int bad = 0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        acc = red_combine(op, acc, partials[t]);
        bad |= flags[t];
    }
    sh[threadIdx.x] = acc;
    shb[threadIdx.x] = bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        unsigned int b = shb[0];
        for (int t = 1; t < (int)blockDim.x; ++t) {
            r = red_combine(op, r, sh[t]);
            b |= shb[t];
        }
        if (op == AC_RMS) r = sqrt(r / count);
        result[0] = r;
        reinterpret_cast<unsigned int *>(result + 1)[0] = b;
    }
}

template <typename R>
static cudaError_t launch_reduce_t(const ReduceLaunch &L, cudaStream_t st, int *launches) {
    PtrPack<const R> pk;
    for (int q = 0; q < NF; ++q) pk.p[q] = static_cast<const R *>(L.f[q]);
    const DevCoefs<R> k = to_dev<R>(L.c, L.ph);
    const long long total = (long long)L.g.nx * L.g.ny * L.g.nz;
    const long long rows = (long long)L.g.ny * L.g.nz;
    long long blocks = (rows + RED_THREADS / 32 - 1) / (RED_THREADS / 32);
    if (blocks > L.blocks) blocks = L.blocks;
    if (blocks < 1) blocks = 1;
    const unsigned nb = (unsigned)blocks;
    // B = curl A uses the handle's stencil order (padded layout: radius <= 3)
    switch (L.c.radius) {
        case 1:
            if (L.g.padded)
                reduce_kernel<R, IdxPadded, 1><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            else
                reduce_kernel<R, IdxPeriodicR<1>, 1><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            break;
        case 2:
            if (L.g.padded)
                reduce_kernel<R, IdxPadded, 2><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            else
                reduce_kernel<R, IdxPeriodicR<2>, 2><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            break;
        case 4:
            reduce_kernel<R, IdxPeriodicR<4>, 4><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            break;
        default:
            if (L.g.padded)
                reduce_kernel<R, IdxPadded><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            else
                reduce_kernel<R, IdxPeriodic><<<nb, RED_THREADS, 0, st>>>(pk, L.g, k, L.op, L.quantity, L.partials, L.flags);
            break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<1, RED_THREADS, 0, st>>>(L.partials, L.flags, (int)blocks, L.op,
                                                   (double)total, L.result);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceLaunch &L, cudaStream_t st, int *launches) {
    if (L.precision == AC_FP64) return launch_reduce_t<double>(L, st, launches);
    return launch_reduce_t<float>(L, st, launches);
}

}  // namespace ac

#ifdef AC_BOUNDS_CHECK
namespace ac {
// Self-test of the checks: two indices are only computed, never used to
// address memory: -5 against an extent of 10 must be recorded (tag 7) and
// redirected to 0, 3 must pass unchanged.
__global__ void bc_selftest_kernel(long long *out) {
    out[0] = AC_BC(-5ll, 10ll, 7u);
    out[1] = AC_BC(3ll, 10ll, 7u);
}
}  // namespace ac
#endif

extern "C" int ac_bounds_check_selftest(long long out[2]) {
    if (!out) return AC_ERR_ARG;
#ifdef AC_BOUNDS_CHECK
    long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(long long));
    if (e == cudaSuccess) {
        ac::bc_selftest_kernel<<<1, 1>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d, 2 * sizeof(long long), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    return e == cudaSuccess ? AC_OK : ac::ac_report_cuda(e);
#else
    out[0] = out[1] = 0;
    return AC_ERR_STATE;
#endif
}

AC_BC_READER(bc_take_aux)
