// ac_reduce_noalloc: the binary64 reduction of ac_reduce for callers that may
// not allocate device memory, with its scratch in a fixed device array.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden,
// e.g. a host application that owns all device memory through its own pool
// and only lends the library its field arrays, or a caller working inside a
// phase of its program in which allocating would synchronise the device or
// fragment a pool it manages.  Such a caller cannot create an ac_handle (which
// allocates work areas) but can still ask for a max, min, sum or rms of the
// state it holds.
//
// Scratch: one binary64 partial and one flag word per z-plane plus the
// result, in the file-scope array below (AC_NOALLOC_MAX_NZ planes; about
// 96 KiB).  Every GPU that loads the library holds it until the process ends.
// All calls share it: a call overwrites every slot it uses before reading it,
// and calls whose work overlaps on the GPU (other streams, other host threads)
// race on it.
#include <stddef.h>
#include <string.h>

#include "reduce.cuh"

namespace ac {

struct NoallocScratch {
    double partial[AC_NOALLOC_MAX_NZ];
    unsigned int flag[AC_NOALLOC_MAX_NZ];
    double result[2];  // value, then the non-finite flag word
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int NOALLOC_THREADS = 256;

// Pass 1: block z reduces z-plane z into partial[z] and flag[z].
template <typename R, class IX>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    reduce_plane_kernel(PtrPack<const R> pk, Geom g, DevCoefs<R> k, int op, int quantity,
                        NoallocScratch *scr) {
    const int z = blockIdx.x;
    const long long plane = (long long)g.nx * g.ny;
    double acc = red_init(op);
    unsigned int bad = 0;
    for (long long t = threadIdx.x; t < plane; t += blockDim.x) {
        const int j = (int)(t / g.nx);
        const int i = (int)(t - (long long)j * g.nx);
        IX ix;
        ix.set_xy(i, j, g);
        ix.set_z(z, g);
        const double v = cell_quantity<R>(pk.p, ix, k, quantity);
        if (!isfinite(v)) bad = 1;
        acc = red_combine(op, acc, op == AC_RMS ? v * v : v);
    }
    __shared__ double sh[NOALLOC_THREADS / 32];
    __shared__ unsigned int shb[NOALLOC_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc = red_combine(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[wid] = acc;
        shb[wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        unsigned int b = shb[0];
        for (int w = 1; w < NOALLOC_THREADS / 32; ++w) {
            r = red_combine(op, r, sh[w]);
            b |= shb[w];
        }
        scr->partial[z] = r;
        scr->flag[z] = b;
    }
}

// Pass 2: one block combines the nz partials in a fixed order.
__global__ void reduce_planes_final_kernel(int nz, int op, double count, NoallocScratch *scr) {
    __shared__ double sh[NOALLOC_THREADS];
    __shared__ unsigned int shb[NOALLOC_THREADS];
    double acc = red_init(op);
    unsigned int bad = 0;
    for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        acc = red_combine(op, acc, scr->partial[t]);
        bad |= scr->flag[t];
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
        scr->result[0] = r;
        reinterpret_cast<unsigned int *>(&scr->result[1])[0] = b;
    }
}

// Device address of the current device's copy of the scratch array.  The
// symbol's host-side name is not a device address, so the runtime is asked,
// with the device current, on every call: the lookup allocates nothing, and an
// address kept from an earlier call could outlive a reset of the device's
// context.
static cudaError_t noalloc_scratch(NoallocScratch **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<NoallocScratch *>(p);
    return cudaSuccess;
}

template <typename R>
static cudaError_t noalloc_launch(const void *const fields[NF], const Geom &g,
                                  const DevCoefs<R> &k, int op, int quantity,
                                  NoallocScratch *scr, cudaStream_t st) {
    PtrPack<const R> pk;
    for (int q = 0; q < NF; ++q) pk.p[q] = static_cast<const R *>(fields[q]);
    if (g.padded)
        reduce_plane_kernel<R, IdxPadded><<<g.nz, NOALLOC_THREADS, 0, st>>>(pk, g, k, op, quantity,
                                                                             scr);
    else
        reduce_plane_kernel<R, IdxPeriodic><<<g.nz, NOALLOC_THREADS, 0, st>>>(pk, g, k, op,
                                                                               quantity, scr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_planes_final_kernel<<<1, NOALLOC_THREADS, 0, st>>>(
        g.nz, op, (double)g.nx * g.ny * g.nz, scr);
    return cudaGetLastError();
}

}  // namespace ac

using namespace ac;

extern "C" int ac_reduce_noalloc(const void *const fields[8], const ac_grid *grid,
                                 const ac_params *params, int op, int quantity, double *out,
                                 void *stream) {
    if (!fields || !out || !valid_grid(grid) || !valid_params(params)) return AC_ERR_ARG;
    if (op < AC_MAX || op > AC_RMS || quantity < 0 || quantity > AC_Q_CFL) return AC_ERR_ARG;
    if (grid->nz > AC_NOALLOC_MAX_NZ) return AC_ERR_ARG;  // one scratch slot per z-plane
    for (int q = 0; q < NF; ++q)
        if (!fields[q]) return AC_ERR_ARG;

    NoallocScratch *scr = nullptr;
    cudaError_t e = noalloc_scratch(&scr);
    if (e != cudaSuccess) return ac_report_cuda(e);
    const Geom g = make_geom(grid->nx, grid->ny, grid->nz, grid->layout);
    const double dx[3] = {grid->lx / grid->nx, grid->ly / grid->ny, grid->lz / grid->nz};
    const StencilCoefs c = make_coefs(dx);
    const PhysConsts ph = make_phys(*params);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (params->precision == AC_FP64)
        e = noalloc_launch<double>(fields, g, to_dev<double>(c, ph), op, quantity, scr, st);
    else
        e = noalloc_launch<float>(fields, g, to_dev<float>(c, ph), op, quantity, scr, st);
    if (e != cudaSuccess) return ac_report_cuda(e);
    double res[2];
    const void *res_dev = reinterpret_cast<const char *>(scr) + offsetof(NoallocScratch, result);
    e = cudaMemcpyAsync(res, res_dev, sizeof res, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ac_report_cuda(e);
    *out = res[0];
    unsigned int flag;
    memcpy(&flag, &res[1], sizeof flag);
    return flag ? AC_ERR_NONFINITE : AC_OK;
}

AC_BC_READER(bc_take_noalloc)
