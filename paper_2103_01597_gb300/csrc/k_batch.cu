// Batched ensemble of independent periodic boxes (uneven sizes, per-box nu and
// eta) advanced by one persistent kernel launch per Runge-Kutta substep.
//
// The paper notes that parameter scans inflate problem sizes (Sec. 4); here a
// scan is a set of small boxes integrated together.  Work items are
// (box, column tile of the box's shape -- 32 x 8 or 16 x 16 --, z range); they
// are sorted by cost (largest first) and taken by persistent CTAs from a device
// counter that a memset node resets before every launch, so the kernel
// boundary is the only cross-CTA synchronisation.  Each item runs the same
// per-cell arithmetic as the single-box binary32 kernel, so every box's result
// is bitwise the single-box result whatever its tile shape.  The three
// substeps of a step can be captured into a CUDA graph; the z extent of the
// items and the tile shape of each box-size class are chosen by a measuring
// autotuner.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "substep_tiled.cuh"

namespace ac {

// One box of the ensemble as the kernel sees it (kernel-parameter space).
struct BatchBox {
    int nx, ny, nz, pad;
    long long off;  // element offset of the box's first field in each pool
    long long n;    // cells of the box (elements per field)
    DevCoefs<float> k;
};

template <typename W>
struct BatchArgs {
    const float *fin;  // state pool read this substep
    float *fout;       // state pool written this substep
    W *w;              // accumulator pool
    const int4 *items; // (box | shape << 16, x0, y0, z0 << 16 | z1)
    unsigned int *counter;
    int nitems;
    int s0;
    W alpha, beta, dt;
    BatchBox box[AC_BATCH_MAX_BOXES];
};

// Argument adapter of one box inside the persistent kernel.
template <typename W>
struct TileBox {
    const BatchArgs<W> &b;
    const BatchBox &x;
    Geom gg;
    __device__ __forceinline__ TileBox(const BatchArgs<W> &b_, const BatchBox &x_) : b(b_), x(x_) {
        gg.nx = x.nx;
        gg.ny = x.ny;
        gg.nz = x.nz;
        gg.padded = 0;
        gg.px = x.nx;
        gg.pxy = (long long)x.nx * x.ny;
        gg.origin = 0;
        gg.elems = x.n;
    }
    __device__ __forceinline__ const float *fin(int q) const { return b.fin + x.off + q * x.n; }
    __device__ __forceinline__ float *fout(int q) const { return b.fout + x.off + q * x.n; }
    __device__ __forceinline__ W *w(int q) const { return b.w + x.off + q * x.n; }
    __device__ __forceinline__ const Geom &g() const { return gg; }
    __device__ __forceinline__ const DevCoefs<float> &k() const { return x.k; }
    __device__ __forceinline__ W alpha() const { return b.alpha; }
    __device__ __forceinline__ W beta() const { return b.beta; }
    __device__ __forceinline__ W dt() const { return b.dt; }
    __device__ __forceinline__ int s0() const { return b.s0; }
    __device__ __forceinline__ int force_on() const { return 0; }
    __device__ __forceinline__ const float2 *ftab() const { return nullptr; }
    __device__ __forceinline__ float amp_e(int) const { return 0.f; }
    __device__ __forceinline__ unsigned long long *cfl_max() const { return nullptr; }
};

// SHAPES: which tile bodies the kernel holds -- AC_TILE_32X8 or AC_TILE_16X16 alone
// (every box on that shape: one body, its own register allocation), or both (2).
template <typename W, int SHAPES>
__global__ void __launch_bounds__(TT_THREADS, 1) batch_substep_kernel(const __grid_constant__ BatchArgs<W> b) {
    extern __shared__ __align__(128) unsigned char bt_smem_raw[];
    __shared__ int item_sh;
    for (;;) {
        if (threadIdx.x == 0 && threadIdx.y == 0) item_sh = (int)atomicAdd(b.counter, 1u);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();  // every thread has read item_sh before it is overwritten
        if (it >= b.nitems) break;
        const int4 wi = b.items[it];
        const TileBox<W> ta(b, b.box[wi.x & 0xffff]);
        if (SHAPES == AC_TILE_16X16 || (SHAPES == 2 && (wi.x >> 16)))
            tiled_body<Tile16x16, W, true, false, false>(ta, wi.y, wi.z, wi.w >> 16, wi.w & 0xffff,
                                                         bt_smem_raw);
        else
            tiled_body<Tile32x8, W, true, false, false>(ta, wi.y, wi.z, wi.w >> 16, wi.w & 0xffff,
                                                        bt_smem_raw);
    }
}

// Dynamic shared memory of the batch kernel: the larger of the two shapes' rings.
template <typename W>
constexpr size_t batch_smem_bytes() {
    return tt_smem_bytes<W, Tile32x8>() > tt_smem_bytes<W, Tile16x16>() ? tt_smem_bytes<W, Tile32x8>()
                                                                        : tt_smem_bytes<W, Tile16x16>();
}

}  // namespace ac

using namespace ac;

static const double B_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double B_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

struct ac_batch {
    int nbox;
    std::vector<ac_box> boxes;
    ac_params common;
    int precision;
    int elem_w;
    cudaStream_t stream;
    std::vector<long long> off, n;
    long long total;  // cells over all boxes
    void *block;      // one allocation: two state pools, w pool
    float *pool[2];
    void *wpool;
    int cur;
    std::vector<DevCoefs<float>> coefs;
    int4 *items_dev;
    int nitems;
    unsigned int *counter;
    int zc;           // z extent of a work item (tuned)
    std::vector<int> shape;  // tile shape of each box (AC_TILE_32X8 / AC_TILE_16X16, tuned)
    int shapes_in_use;       // bit 0: some box on 32 x 8, bit 1: some box on 16 x 16
    float tune_ms[2];        // last tuning: full step with the default split, and tuned
    int ctas;         // persistent CTAs
    int next_s;
    unsigned long long step;
    int graph_on;
    cudaStream_t cap_stream;
    cudaGraphExec_t exec[2];
    double graph_dt[2];
    double *stage;
    size_t stage_elems;
    double *partials, *result_dev, *result_host;
    unsigned int *flags;
    unsigned long long launches;
};

#define BCK(call)                                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return ac_report_cuda(e_); \
    } while (0)

// Work items for z extent zc and the boxes' tile shapes; cost = planes staged
// (z extent + 6), the same for every full tile of either shape.
static int build_items(ac_batch *b, int zc) {
    std::vector<int4> items;
    std::vector<long long> cost;
    for (int bx = 0; bx < b->nbox; ++bx) {
        const ac_box &x = b->boxes[bx];
        const int sh = b->shape[bx];
        const int TX = sh ? Tile16x16::TX : Tile32x8::TX, TY = sh ? Tile16x16::TY : Tile32x8::TY;
        const int z = std::min(zc, x.nz);
        for (int z0 = 0; z0 < x.nz; z0 += z)
            for (int y0 = 0; y0 < x.ny; y0 += TY)
                for (int x0 = 0; x0 < x.nx; x0 += TX) {
                    const int z1 = std::min(z0 + z, x.nz);
                    items.push_back(make_int4(bx | (sh << 16), x0, y0, (z0 << 16) | z1));
                    cost.push_back((long long)(z1 - z0 + 6) * std::min(TY, x.ny - y0) *
                                   std::min(TX, x.nx - x0));
                }
    }
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<int4> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    if (b->items_dev) {
        BCK(cudaStreamSynchronize(b->stream));
        cudaFree(b->items_dev);
        b->items_dev = nullptr;
    }
    BCK(cudaMalloc(&b->items_dev, sizeof(int4) * sorted.size()));
    BCK(cudaMemcpy(b->items_dev, sorted.data(), sizeof(int4) * sorted.size(),
                   cudaMemcpyHostToDevice));
    b->nitems = (int)sorted.size();
    b->zc = zc;
    b->shapes_in_use = 0;
    for (int v : b->shape) b->shapes_in_use |= v == AC_TILE_16X16 ? 2 : 1;
    for (int c = 0; c < 2; ++c)
        if (b->exec[c]) {
            cudaGraphExecDestroy(b->exec[c]);
            b->exec[c] = nullptr;
        }
    return AC_OK;
}

template <typename W>
static cudaError_t launch_batch_t(ac_batch *b, double dt, int s, int cur, cudaStream_t st) {
    BatchArgs<W> a;
    a.fin = b->pool[cur];
    a.fout = b->pool[1 - cur];
    a.w = static_cast<W *>(b->wpool);
    a.items = b->items_dev;
    a.counter = b->counter;
    a.nitems = b->nitems;
    a.s0 = s == 0;
    a.alpha = (W)B_ALPHA[s];
    a.beta = (W)B_BETA[s];
    a.dt = (W)dt;
    for (int i = 0; i < b->nbox; ++i) {
        a.box[i].nx = b->boxes[i].nx;
        a.box[i].ny = b->boxes[i].ny;
        a.box[i].nz = b->boxes[i].nz;
        a.box[i].pad = 0;
        a.box[i].off = b->off[i];
        a.box[i].n = b->n[i];
        a.box[i].k = b->coefs[i];
    }
    cudaError_t e = cudaMemsetAsync(b->counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const size_t smem = batch_smem_bytes<W>();
    // one body when every box has the same shape
    auto k = b->shapes_in_use == 1 ? batch_substep_kernel<W, AC_TILE_32X8>
             : b->shapes_in_use == 2 ? batch_substep_kernel<W, AC_TILE_16X16>
                                     : batch_substep_kernel<W, 2>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<b->ctas, dim3(32, 8, 1), smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_batch(ac_batch *b, double dt, int s, int cur, cudaStream_t st) {
    if (b->precision == AC_FP32) return launch_batch_t<float>(b, dt, s, cur, st);
    return launch_batch_t<double>(b, dt, s, cur, st);
}

static void free_batch(ac_batch *b) {
    for (int c = 0; c < 2; ++c)
        if (b->exec[c]) cudaGraphExecDestroy(b->exec[c]);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->block) cudaFree(b->block);
    if (b->items_dev) cudaFree(b->items_dev);
    if (b->counter) cudaFree(b->counter);
    if (b->stage) cudaFree(b->stage);
    if (b->partials) cudaFree(b->partials);
    if (b->flags) cudaFree(b->flags);
    if (b->result_dev) cudaFree(b->result_dev);
    if (b->result_host) cudaFreeHost(b->result_host);
}

extern "C" int ac_batch_init(ac_batch **out, int nbox, const ac_box *boxes, const ac_params *common,
                             void *stream) {
    if (!out || !boxes || !common || nbox < 1 || nbox > AC_BATCH_MAX_BOXES) return AC_ERR_ARG;
    *out = nullptr;
    if (common->precision != AC_FP32 && common->precision != AC_FP32_W64) return AC_ERR_ARG;
    if (common->force_amp != 0.0) return AC_ERR_ARG;
    if (!(common->cs0 > 0) || !(common->gamma > 1.0) || !(common->cp > 0) ||
        !isfinite(common->lnrho0))
        return AC_ERR_ARG;
    for (int i = 0; i < nbox; ++i) {
        const ac_box &x = boxes[i];
        if (x.nx < 1 || x.ny < 1 || x.nz < 1 || x.nx % 4 || x.nx > 4096 || x.ny > 4096 ||
            x.nz > 4096)
            return AC_ERR_ARG;
        if (!(x.lx > 0) || !(x.ly > 0) || !(x.lz > 0) || !(x.nu >= 0) || !(x.eta >= 0) ||
            !isfinite(x.nu) || !isfinite(x.eta))
            return AC_ERR_ARG;
    }
    ac_batch *b = new (std::nothrow) ac_batch();
    if (!b) return AC_ERR_OOM;
    b->nbox = nbox;
    b->boxes.assign(boxes, boxes + nbox);
    b->common = *common;
    b->precision = common->precision;
    b->elem_w = common->precision == AC_FP32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(stream);
    long long total = 0;
    for (int i = 0; i < nbox; ++i) {
        const ac_box &x = boxes[i];
        b->off.push_back(8 * total);
        b->n.push_back((long long)x.nx * x.ny * x.nz);
        total += (long long)x.nx * x.ny * x.nz;
        ac_params p = *common;
        p.nu = x.nu;
        p.eta = x.eta;
        const double dx[3] = {x.lx / x.nx, x.ly / x.ny, x.lz / x.nz};
        b->coefs.push_back(to_dev<float>(make_coefs(dx), make_phys(p)));
    }
    b->total = total;
    const size_t fbytes = (size_t)8 * total * sizeof(float);
    const size_t wbytes = (size_t)8 * total * b->elem_w;
    cudaError_t e = cudaMalloc(&b->block, 2 * fbytes + wbytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->block, 0, 2 * fbytes + wbytes, b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->partials, sizeof(double) * reduce_max_blocks());
    if (e == cudaSuccess) e = cudaMalloc(&b->flags, sizeof(unsigned int) * reduce_max_blocks());
    if (e == cudaSuccess) e = cudaMalloc(&b->result_dev, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->result_host, 2 * sizeof(double));
    int dev = 0, sms = 152, occ = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const size_t smem = b->precision == AC_FP32 ? batch_smem_bytes<float>() : batch_smem_bytes<double>();
        if (b->precision == AC_FP32) {
            e = cudaFuncSetAttribute(batch_substep_kernel<float, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_substep_kernel<float, 2>,
                                                                  TT_THREADS, smem);
        } else {
            e = cudaFuncSetAttribute(batch_substep_kernel<double, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &occ, batch_substep_kernel<double, 2>, TT_THREADS, smem);
        }
    }
    if (e != cudaSuccess) {
        int rc = ac_report_cuda(e);
        free_batch(b);
        delete b;
        return rc;
    }
    b->pool[0] = static_cast<float *>(b->block);
    b->pool[1] = reinterpret_cast<float *>(static_cast<char *>(b->block) + fbytes);
    b->wpool = static_cast<char *>(b->block) + 2 * fbytes;
    b->ctas = sms * (occ < 1 ? 1 : occ);
    b->shape.assign(nbox, AC_TILE_32X8);
    int rc = build_items(b, 64);
    if (rc) {
        free_batch(b);
        delete b;
        return rc;
    }
    *out = b;
    return AC_OK;
}

extern "C" int ac_batch_quit(ac_batch *b) {
    if (!b) return AC_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return AC_OK;
}

static int batch_stage(ac_batch *b, size_t need) {
    if (b->stage_elems >= need) return AC_OK;
    if (b->stage) {
        BCK(cudaStreamSynchronize(b->stream));
        cudaFree(b->stage);
        b->stage = nullptr;
        b->stage_elems = 0;
    }
    BCK(cudaMalloc(&b->stage, need * sizeof(double)));
    b->stage_elems = need;
    return AC_OK;
}

static Geom box_geom(const ac_box &x) { return make_geom(x.nx, x.ny, x.nz, AC_LAYOUT_PERIODIC); }

static int batch_copy(ac_batch *b, int box, int field, double *host, int to_device, int w_arr) {
    if (!b || !host || box < 0 || box >= b->nbox || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    const Geom g = box_geom(b->boxes[box]);
    const long long n = b->n[box];
    int rc = batch_stage(b, (size_t)n);
    if (rc) return rc;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    for (int q = q0; q < q1; ++q) {
        double *h = host + (field == AC_ALL ? (size_t)q * n : 0);
        void *dev;
        int es;
        if (w_arr) {
            es = b->elem_w;
            dev = static_cast<char *>(b->wpool) + (size_t)(b->off[box] + q * n) * es;
        } else {
            es = 4;
            dev = b->pool[b->cur] + b->off[box] + q * n;
        }
        if (to_device) {
            BCK(cudaMemcpyAsync(b->stage, h, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
            BCK(launch_scatter(b->stage, dev, es, g, 0, g.nz, b->stream));
        } else {
            BCK(launch_gather(dev, es, g, 0, g.nz, b->stage, b->stream));
            BCK(cudaMemcpyAsync(h, b->stage, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        }
        b->launches++;
    }
    if (!to_device) BCK(cudaStreamSynchronize(b->stream));
    else if (!w_arr) b->next_s = 0;
    return AC_OK;
}

// Host float32 <-> one box's state: the pool holds binary32 fields, a box's
// eight arrays back to back, so each call is one copy.
static int batch_copy_f32(ac_batch *b, int box, int field, float *host, int to_device) {
    if (!b || !host || box < 0 || box >= b->nbox || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    const long long n = b->n[box];
    float *dev = b->pool[b->cur] + b->off[box] + (field == AC_ALL ? 0 : (long long)field * n);
    const size_t bytes = sizeof(float) * (size_t)n * (field == AC_ALL ? NF : 1);
    if (to_device) {
        BCK(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, b->stream));
        b->next_s = 0;
    } else {
        BCK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
    }
    return AC_OK;
}

extern "C" int ac_batch_load_f32(ac_batch *b, int box, int field, const float *host) {
    return batch_copy_f32(b, box, field, const_cast<float *>(host), 1);
}
extern "C" int ac_batch_store_f32(ac_batch *b, int box, int field, float *host) {
    return batch_copy_f32(b, box, field, host, 0);
}

extern "C" int ac_batch_load(ac_batch *b, int box, int field, const double *host) {
    return batch_copy(b, box, field, const_cast<double *>(host), 1, 0);
}
extern "C" int ac_batch_store(ac_batch *b, int box, int field, double *host) {
    return batch_copy(b, box, field, host, 0, 0);
}
extern "C" int ac_batch_load_w(ac_batch *b, int box, int field, const double *host) {
    return batch_copy(b, box, field, const_cast<double *>(host), 1, 1);
}
extern "C" int ac_batch_store_w(ac_batch *b, int box, int field, double *host) {
    return batch_copy(b, box, field, host, 0, 1);
}

extern "C" int ac_batch_integrate_substep(ac_batch *b, double dt, int s) {
    AC_RANGE("ac_batch_integrate_substep");
    if (!b || s < 0 || s > 2 || !isfinite(dt)) return AC_ERR_ARG;
    if (s != b->next_s) return AC_ERR_STATE;
    BCK(launch_batch(b, dt, s, b->cur, b->stream));
    b->launches++;
    b->cur = 1 - b->cur;
    b->next_s = (s + 1) % 3;
    if (s == 2) b->step++;
    return AC_OK;
}

// Capture the three substeps of a step that starts from state pool `cur`.
static int capture_step(ac_batch *b, double dt, int cur) {
    if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    if (b->exec[cur]) {
        cudaGraphExecDestroy(b->exec[cur]);
        b->exec[cur] = nullptr;
    }
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int c = cur;
    for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
        e = launch_batch(b, dt, s, c, b->cap_stream);
        c = 1 - c;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[cur], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return ac_report_cuda(e);
    b->graph_dt[cur] = dt;
    return AC_OK;
}

extern "C" int ac_batch_set_graph(ac_batch *b, int enable) {
    if (!b) return AC_ERR_ARG;
    b->graph_on = enable != 0;
    return AC_OK;
}

extern "C" int ac_batch_integrate_step(ac_batch *b, double dt) {
    AC_RANGE("ac_batch_integrate_step");
    if (!b || !isfinite(dt)) return AC_ERR_ARG;
    if (b->next_s != 0) return AC_ERR_STATE;
    if (!b->graph_on) {
        for (int s = 0; s < 3; ++s) {
            int rc = ac_batch_integrate_substep(b, dt, s);
            if (rc) return rc;
        }
        return AC_OK;
    }
    if (!b->exec[b->cur] || b->graph_dt[b->cur] != dt) {
        int rc = capture_step(b, dt, b->cur);
        if (rc) return rc;
    }
    BCK(cudaGraphLaunch(b->exec[b->cur], b->stream));
    b->launches += 3;
    b->cur = 1 - b->cur;  // three substeps: an odd number of pool swaps
    b->step++;
    return AC_OK;
}

// Autotuner.  A candidate split (z extent, tile shape per box) is timed over a
// whole step (substeps 0, 1, 2: substeps 1 and 2 also read the accumulator),
// from the same state each time: the current state pool is copied aside once
// and put back before every timed step and at the end (a step at a step
// boundary rewrites w before reading it, so w needs no copy).  Search: every z
// extent with all boxes on one shape, for both shapes; then, for each box-size
// class (boxes of equal nx, ny; largest total first), the other shape, kept if
// the step gets faster by more than the noise margin.
static const int TUNE_ZC[5] = {8, 16, 32, 64, 128};
static const float TUNE_MARGIN = 0.003f;  // relative gain a class change must beat

static std::string batch_signature(const ac_batch *b) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, dev);
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the box sizes
    for (const ac_box &x : b->boxes) {
        const int v[3] = {x.nx, x.ny, x.nz};
        for (int a = 0; a < 3; ++a) {
            h ^= (uint64_t)(unsigned)v[a];
            h *= 1099511628211ull;
        }
    }
    char buf[256];
    snprintf(buf, sizeof buf, "%s|sm%d|p%d|n%d|%016llx", prop.name, prop.multiProcessorCount,
             b->precision, b->nbox, (unsigned long long)h);
    std::string s(buf);
    for (char &c : s)
        if (c == ' ' || c == '"' || c == '\\') c = '_';
    return s;
}

// Shortest of `reps` steps (after one untimed) from the saved state `save`.
static int time_step(ac_batch *b, double dt, const float *save, size_t bytes, int reps, cudaEvent_t e0,
                     cudaEvent_t e1, float *ms_out) {
    float tmin = 1e30f;
    for (int r = 0; r <= reps; ++r) {
        BCK(cudaMemcpyAsync(b->pool[b->cur], save, bytes, cudaMemcpyDeviceToDevice, b->stream));
        BCK(cudaEventRecord(e0, b->stream));
        int c = b->cur;
        for (int s = 0; s < 3; ++s, c = 1 - c) BCK(launch_batch(b, dt, s, c, b->stream));
        BCK(cudaEventRecord(e1, b->stream));
        BCK(cudaEventSynchronize(e1));
        b->launches += 3;
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0 && ms < tmin) tmin = ms;
    }
    *ms_out = tmin;
    return AC_OK;
}

// One entry per line of the cache file, the file a JSON object:
//   {
//     "<signature>": {"zc": 64, "tiles": "0110...", "ms_default": 3.6, "ms_tuned": 3.4},
//     ...
//   }
// ("tiles": one digit per box, AC_TILE_32X8 = 0, AC_TILE_16X16 = 1).
struct CacheEntry {
    std::string key, tiles;
    int zc;
    float ms[2];
};

static bool parse_entry(const char *line, CacheEntry *e) {
    char key[512], tiles[AC_BATCH_MAX_BOXES + 1];
    int zc = 0;
    float m0 = 0.f, m1 = 0.f;
    const int got = sscanf(line, " \"%511[^\"]\": {\"zc\": %d, \"tiles\": \"%128[01]\", \"ms_default\": %f, "
                           "\"ms_tuned\": %f", key, &zc, tiles, &m0, &m1);
    if (got < 3 || zc <= 0) return false;
    e->key = key;
    e->tiles = tiles;
    e->zc = zc;
    e->ms[0] = got >= 4 ? m0 : 0.f;
    e->ms[1] = got >= 5 ? m1 : 0.f;
    return true;
}

// Read the entries; false if the file holds anything this format does not
// (then it is never rewritten).
static bool read_cache(const char *path, std::vector<CacheEntry> *out) {
    FILE *f = fopen(path, "r");
    if (!f) return true;  // no file yet
    char line[1024];
    bool ok = true;
    while (fgets(line, sizeof line, f)) {
        CacheEntry e;
        if (parse_entry(line, &e)) {
            out->push_back(e);
            continue;
        }
        // besides entries, only blank lines and the object's own braces
        std::string t;
        for (const char *p = line; *p; ++p)
            if (*p != ' ' && *p != '\t' && *p != '\n' && *p != '\r') t.push_back(*p);
        if (!t.empty() && t != "{" && t != "}") ok = false;
    }
    fclose(f);
    return ok;
}

static void write_cache(const char *path, const std::vector<CacheEntry> &es) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    for (size_t i = 0; i < es.size(); ++i)
        fprintf(f, "  \"%s\": {\"zc\": %d, \"tiles\": \"%s\", \"ms_default\": %.4f, \"ms_tuned\": %.4f}%s\n",
                es[i].key.c_str(), es[i].zc, es[i].tiles.c_str(), es[i].ms[0], es[i].ms[1],
                i + 1 < es.size() ? "," : "");
    fprintf(f, "}\n");
    const bool good = fclose(f) == 0;
    if (good) rename(tmp.c_str(), path);
    else remove(tmp.c_str());
}

static int set_tiling(ac_batch *b, int zc, const std::vector<int> &shape) {
    b->shape = shape;
    return build_items(b, zc);
}

static int tune_measure(ac_batch *b, double dt) {
    const size_t bytes = (size_t)8 * b->total * sizeof(float);
    float *save = nullptr;
    BCK(cudaMalloc(&save, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMemcpyAsync(save, b->pool[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    int rc = ce == cudaSuccess ? AC_OK : ac_report_cuda(ce);
    const int reps = 3;
    std::vector<int> best_shape(b->nbox, AC_TILE_32X8);
    int best_zc = 64;
    float best = 1e30f, t = 0.f;
    if (rc == AC_OK) rc = set_tiling(b, 64, best_shape);
    if (rc == AC_OK) rc = time_step(b, dt, save, bytes, reps, e0, e1, &t);
    if (rc == AC_OK) b->tune_ms[0] = t;
    for (int sh = 0; sh < 2 && rc == AC_OK; ++sh)
        for (int c = 0; c < 5 && rc == AC_OK; ++c) {
            const std::vector<int> all(b->nbox, sh);
            rc = set_tiling(b, TUNE_ZC[c], all);
            if (rc == AC_OK) rc = time_step(b, dt, save, bytes, reps, e0, e1, &t);
            if (rc == AC_OK && t < best) {
                best = t;
                best_zc = TUNE_ZC[c];
                best_shape = all;
            }
        }
    // box-size classes, largest total first
    std::vector<std::pair<long long, std::pair<int, int>>> classes;
    for (const ac_box &x : b->boxes) {
        bool seen = false;
        for (auto &c : classes)
            if (c.second.first == x.nx && c.second.second == x.ny) {
                c.first += (long long)x.nx * x.ny * x.nz;
                seen = true;
            }
        if (!seen) classes.push_back({(long long)x.nx * x.ny * x.nz, {x.nx, x.ny}});
    }
    std::stable_sort(classes.begin(), classes.end(),
                     [](const auto &p, const auto &q) { return p.first > q.first; });
    for (size_t k = 0; k < classes.size() && classes.size() > 1 && rc == AC_OK; ++k) {
        std::vector<int> trial = best_shape;
        for (int i = 0; i < b->nbox; ++i)
            if (b->boxes[i].nx == classes[k].second.first && b->boxes[i].ny == classes[k].second.second)
                trial[i] = 1 - trial[i];
        rc = set_tiling(b, best_zc, trial);
        if (rc == AC_OK) rc = time_step(b, dt, save, bytes, reps, e0, e1, &t);
        if (rc == AC_OK && t < best * (1.f - TUNE_MARGIN)) {
            best = t;
            best_shape = trial;
        }
    }
    if (rc == AC_OK) rc = set_tiling(b, best_zc, best_shape);
    if (rc == AC_OK) b->tune_ms[1] = best;
    // the state as it was
    ce = cudaMemcpyAsync(b->pool[b->cur], save, bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (rc == AC_OK && ce != cudaSuccess) rc = ac_report_cuda(ce);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    return rc;
}

extern "C" int ac_batch_tune(ac_batch *b, double dt, const char *cache_path, int *zc_out) {
    if (!b || !isfinite(dt)) return AC_ERR_ARG;
    if (b->next_s != 0) return AC_ERR_STATE;
    const std::string sig = batch_signature(b);
    std::vector<CacheEntry> cache;
    const bool writable = cache_path ? read_cache(cache_path, &cache) : false;
    for (const CacheEntry &e : cache)
        if (e.key == sig && (int)e.tiles.size() == b->nbox) {
            std::vector<int> shape(b->nbox);
            for (int i = 0; i < b->nbox; ++i) shape[i] = e.tiles[i] - '0';
            int rc = set_tiling(b, e.zc, shape);
            if (rc) return rc;
            b->tune_ms[0] = e.ms[0];
            b->tune_ms[1] = e.ms[1];
            if (zc_out) *zc_out = e.zc;
            return AC_OK;
        }
    int rc = tune_measure(b, dt);
    if (rc) return rc;
    if (cache_path && writable) {
        CacheEntry e;
        e.key = sig;
        e.zc = b->zc;
        for (int i = 0; i < b->nbox; ++i) e.tiles.push_back((char)('0' + b->shape[i]));
        e.ms[0] = b->tune_ms[0];
        e.ms[1] = b->tune_ms[1];
        cache.push_back(e);
        write_cache(cache_path, cache);
    }
    if (zc_out) *zc_out = b->zc;
    return AC_OK;
}

extern "C" int ac_batch_set_tiling(ac_batch *b, int zc, const int *shapes) {
    if (!b || zc < 1 || zc > 4096) return AC_ERR_ARG;
    std::vector<int> shape(b->nbox, AC_TILE_32X8);
    if (shapes)
        for (int i = 0; i < b->nbox; ++i) {
            if (shapes[i] != AC_TILE_32X8 && shapes[i] != AC_TILE_16X16) return AC_ERR_ARG;
            shape[i] = shapes[i];
        }
    return set_tiling(b, zc, shape);
}

extern "C" int ac_batch_get_tiling(const ac_batch *b, int *zc, int *shapes, float tune_ms[2]) {
    if (!b) return AC_ERR_ARG;
    if (zc) *zc = b->zc;
    if (shapes)
        for (int i = 0; i < b->nbox; ++i) shapes[i] = b->shape[i];
    if (tune_ms) {
        tune_ms[0] = b->tune_ms[0];
        tune_ms[1] = b->tune_ms[1];
    }
    return AC_OK;
}

extern "C" int ac_batch_reduce(ac_batch *b, int box, int op, int quantity, double *out) {
    if (!b || !out || box < 0 || box >= b->nbox || op < AC_MAX || op > AC_RMS || quantity < 0 ||
        quantity > AC_Q_CFL)
        return AC_ERR_ARG;
    ReduceLaunch L;
    L.precision = AC_FP32;
    L.g = box_geom(b->boxes[box]);
    for (int q = 0; q < NF; ++q) L.f[q] = b->pool[b->cur] + b->off[box] + q * b->n[box];
    const ac_box &x = b->boxes[box];
    const double dx[3] = {x.lx / x.nx, x.ly / x.ny, x.lz / x.nz};
    ac_params p = b->common;
    p.nu = x.nu;
    p.eta = x.eta;
    L.c = make_coefs(dx);
    L.ph = make_phys(p);
    L.op = op;
    L.quantity = quantity;
    L.partials = b->partials;
    L.flags = b->flags;
    L.result = b->result_dev;
    L.blocks = reduce_max_blocks();
    int nl = 0;
    BCK(launch_reduce(L, b->stream, &nl));
    b->launches += nl;
    BCK(cudaMemcpyAsync(b->result_host, b->result_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    *out = b->result_host[0];
    unsigned int flag;
    memcpy(&flag, &b->result_host[1], sizeof flag);
    return flag ? AC_ERR_NONFINITE : AC_OK;
}

extern "C" int ac_batch_info(const ac_batch *b, long long *cells, int *items, int *zc, int *ctas,
                             unsigned long long *launches) {
    if (!b) return AC_ERR_ARG;
    if (cells) *cells = b->total;
    if (items) *items = b->nitems;
    if (zc) *zc = b->zc;
    if (ctas) *ctas = b->ctas;
    if (launches) *launches = b->launches;
    return AC_OK;
}

AC_BC_READER(bc_take_batch)
