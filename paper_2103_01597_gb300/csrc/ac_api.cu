// C-ABI implementation of libac.so (declarations and contracts in include/ac.h).
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ac_internal.h"

namespace ac {
cudaError_t launch_substep_f64(const SubstepLaunch &L, cudaStream_t st, int *launches);
cudaError_t launch_substep_f32(const SubstepLaunch &L, cudaStream_t st, int *launches);
cudaError_t launch_substep_f32w64(const SubstepLaunch &L, cudaStream_t st, int *launches);
}  // namespace ac

using namespace ac;

// Williamson (1980) third-order 2N-storage coefficients (Sec. 4 names the scheme).
static const double RK_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

static thread_local char g_cuda_msg[256] = "";

static int cuda_fail(cudaError_t e) {
    snprintf(g_cuda_msg, sizeof g_cuda_msg, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    // the error is reported through the return code: clear the runtime's
    // per-thread last error so that the caller's next, unrelated CUDA call
    // (an allocation in the application, say) does not find it
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA;
}

int ac::ac_report_cuda(cudaError_t e) { return cuda_fail(e); }

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

struct ac_handle {
    ac_grid grid;
    ac_params params;
    Geom g;
    StencilCoefs coefs;
    PhysConsts phys;
    cudaStream_t stream;
    int elem_f, elem_w;  // bytes per element of state and accumulator arrays
    void *state[2][NF];  // alternating state buffers
    void *w[NF];
    int cur;             // index of the current state
    int have_buffers;
    void *owned_block;   // library-owned state allocation (NULL if bound)
    double2 *ftab;       // forcing tables (double2 then float2)
    double *partials;
    unsigned int *flags;
    double *result_dev;  // [value, flag word]
    double *result_host; // page-locked copy of result_dev
    unsigned long long *cfl_dev;  // max CFL speed of the last substep-0 input (bits of a double)
    int stencil_mode;             // AC_STENCIL_*
    long long *fx_block;          // int64 copies of the fields (integer stencil sums)
    unsigned long long *fx_stats; // per-field extremes (16 words) of the substep's input
    void *fx_plan;                // device plan of the integer-sum path (mode, scales)
    double *stage;       // float64 staging for load/store
    size_t stage_elems;
    int next_s;
    unsigned long long step;
    int force_manual;
    int force_k[3];
    double force_e[3];
    double force_phi;
    int ftab_dirty;
    int ftab_valid;
    unsigned long long ftab_step;  // step whose draw the tables hold (per-step draw mode)
    unsigned long long launches;
    // kernel timing (ac_set_kernel_timing): three events per recorded substep
    int timing;
    int nrec;
    cudaEvent_t *tev;  // [AC_TIMING_MAX][3]: start, after preparation, after the substep
    int trec_s[AC_TIMING_MAX];
};

extern "C" const char *ac_strerror(int code) {
    switch (code) {
        case AC_OK: return "AC_OK: success";
        case AC_ERR_ARG: return "AC_ERR_ARG: invalid argument";
        case AC_ERR_CUDA: return "AC_ERR_CUDA: CUDA runtime error";
        case AC_ERR_OOM: return "AC_ERR_OOM: out of memory";
        case AC_ERR_NONFINITE: return "AC_ERR_NONFINITE: non-finite value met";
        case AC_ERR_TIMEOUT: return "AC_ERR_TIMEOUT: bounded device wait ran out";
        case AC_ERR_STATE: return "AC_ERR_STATE: call out of order";
        default: return "unknown ac error code";
    }
}

extern "C" const char *ac_last_cuda_error(void) { return g_cuda_msg; }

int ac::valid_grid(const ac_grid *g) {
    if (!g) return 0;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return 0;
    if (!(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0)) return 0;
    if (!isfinite(g->lx) || !isfinite(g->ly) || !isfinite(g->lz)) return 0;
    if (g->layout != AC_LAYOUT_PERIODIC && g->layout != AC_LAYOUT_PADDED) return 0;
    // 64-bit cell counts; keep every per-axis index and padded extent in int range.
    if (g->nx > (1 << 24) || g->ny > (1 << 24) || g->nz > (1 << 24)) return 0;
    return 1;
}

int ac::valid_params(const ac_params *p) {
    if (!p) return 0;
    const double v[7] = {p->nu, p->eta, p->cs0, p->gamma, p->cp, p->lnrho0, p->force_amp};
    for (int i = 0; i < 7; ++i)
        if (!isfinite(v[i])) return 0;
    if (p->nu < 0 || p->eta < 0 || p->cs0 <= 0 || p->gamma <= 1.0 || p->cp <= 0) return 0;
    if (p->precision != AC_FP64 && p->precision != AC_FP32 && p->precision != AC_FP32_W64)
        return 0;
    return 1;
}

static void free_timing(ac_handle *h) {
    if (!h->tev) return;
    for (int i = 0; i < 3 * AC_TIMING_MAX; ++i)
        if (h->tev[i]) cudaEventDestroy(h->tev[i]);
    free(h->tev);
    h->tev = nullptr;
}

static void free_handle_memory(ac_handle *h) {
    free_timing(h);
    if (h->owned_block) cudaFree(h->owned_block);
    if (h->ftab) cudaFree(h->ftab);
    if (h->partials) cudaFree(h->partials);
    if (h->flags) cudaFree(h->flags);
    if (h->result_dev) cudaFree(h->result_dev);
    if (h->result_host) cudaFreeHost(h->result_host);
    if (h->stage) cudaFree(h->stage);
    if (h->cfl_dev) cudaFree(h->cfl_dev);
    if (h->fx_block) cudaFree(h->fx_block);
    if (h->fx_stats) cudaFree(h->fx_stats);
    if (h->fx_plan) cudaFree(h->fx_plan);
}

extern "C" int ac_init(ac_handle **out, const ac_grid *grid, const ac_params *params,
                       void *stream) {
    if (!out || !valid_grid(grid) || !valid_params(params)) return AC_ERR_ARG;
    *out = nullptr;
    ac_handle *h = new (std::nothrow) ac_handle();
    if (!h) return AC_ERR_OOM;
    h->grid = *grid;
    h->params = *params;
    h->g = make_geom(grid->nx, grid->ny, grid->nz, grid->layout);
    const double dx[3] = {grid->lx / grid->nx, grid->ly / grid->ny, grid->lz / grid->nz};
    h->coefs = make_coefs(dx, 3);
    h->phys = make_phys(*params);
    h->stream = static_cast<cudaStream_t>(stream);
    h->elem_f = params->precision == AC_FP64 ? 8 : 4;
    h->elem_w = params->precision == AC_FP32 ? 4 : 8;
    const int ntab = grid->nx + grid->ny + grid->nz;
    cudaError_t e = cudaMalloc(&h->ftab, (size_t)ntab * (sizeof(double2) + sizeof(float2)));
    if (e == cudaSuccess) e = cudaMalloc(&h->partials, sizeof(double) * reduce_max_blocks());
    if (e == cudaSuccess) e = cudaMalloc(&h->flags, sizeof(unsigned int) * reduce_max_blocks());
    if (e == cudaSuccess) e = cudaMalloc(&h->result_dev, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h->result_host, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->cfl_dev, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->cfl_dev, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        int rc = cuda_fail(e);
        free_handle_memory(h);
        delete h;
        return rc;
    }
    *out = h;
    return AC_OK;
}

extern "C" int ac_quit(ac_handle *h) {
    if (!h) return AC_OK;
    cudaStreamSynchronize(h->stream);
    free_handle_memory(h);
    delete h;
    return AC_OK;
}

extern "C" int ac_set_stream(ac_handle *h, void *stream) {
    if (!h) return AC_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return AC_OK;
}

extern "C" int ac_field_elems(const ac_handle *h, size_t *elems) {
    if (!h || !elems) return AC_ERR_ARG;
    *elems = (size_t)h->g.elems;
    return AC_OK;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Allocate the library-owned state on first use (zero-filled).
static int ensure_state(ac_handle *h) {
    if (h->have_buffers) return AC_OK;
    const size_t nf = align_up((size_t)h->g.elems * h->elem_f, 256);
    const size_t nw = align_up((size_t)h->g.elems * h->elem_w, 256);
    const size_t total = 2 * NF * nf + NF * nw;
    void *blk = nullptr;
    CK(cudaMalloc(&blk, total));
    cudaError_t e = cudaMemsetAsync(blk, 0, total, h->stream);
    if (e != cudaSuccess) {
        cudaFree(blk);
        return cuda_fail(e);
    }
    char *p = static_cast<char *>(blk);
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < NF; ++q) {
            h->state[b][q] = p;
            p += nf;
        }
    for (int q = 0; q < NF; ++q) {
        h->w[q] = p;
        p += nw;
    }
    h->owned_block = blk;
    h->have_buffers = 1;
    h->cur = 0;
    return AC_OK;
}

extern "C" int ac_bind_buffers(ac_handle *h, void *const dev_ptrs[24]) {
    if (!h || !dev_ptrs) return AC_ERR_ARG;
    for (int i = 0; i < 24; ++i)
        if (!dev_ptrs[i] || ((uintptr_t)dev_ptrs[i] & 15u)) return AC_ERR_ARG;
    if (h->owned_block) {
        CK(cudaStreamSynchronize(h->stream));
        cudaFree(h->owned_block);
        h->owned_block = nullptr;
    }
    for (int q = 0; q < NF; ++q) {
        h->state[0][q] = dev_ptrs[q];
        h->state[1][q] = dev_ptrs[NF + q];
        h->w[q] = dev_ptrs[2 * NF + q];
    }
    h->cur = 0;
    h->have_buffers = 1;
    return AC_OK;
}

static int ensure_stage(ac_handle *h, size_t *planes) {
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    const size_t want_elems = (size_t)1 << 25;  // 256 MiB of float64 at most
    size_t np = want_elems / plane;
    if (np < 1) np = 1;
    if (np > (size_t)h->g.nz) np = (size_t)h->g.nz;
    const size_t need = np * plane;
    if (h->stage_elems < need) {
        if (h->stage) {
            CK(cudaStreamSynchronize(h->stream));
            cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_elems = 0;
        }
        CK(cudaMalloc(&h->stage, need * sizeof(double)));
        h->stage_elems = need;
    }
    *planes = np;
    return AC_OK;
}

// Host float64 (unpadded) -> device array `dst` with element size `es`.
static int load_array(ac_handle *h, void *dst, int es, const double *src) {
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    if (es == 8 && !h->g.padded) {
        CK(cudaMemcpyAsync(dst, src, plane * h->g.nz * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
        return AC_OK;
    }
    size_t np;
    int rc = ensure_stage(h, &np);
    if (rc) return rc;
    for (size_t z0 = 0; z0 < (size_t)h->g.nz; z0 += np) {
        const size_t nzc = (z0 + np <= (size_t)h->g.nz) ? np : (size_t)h->g.nz - z0;
        CK(cudaMemcpyAsync(h->stage, src + z0 * plane, nzc * plane * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream));
        CK(launch_scatter(h->stage, dst, es, h->g, (int)z0, (int)nzc, h->stream));
        h->launches++;
    }
    return AC_OK;
}

static int store_array(ac_handle *h, const void *src, int es, double *dst) {
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    if (es == 8 && !h->g.padded) {
        CK(cudaMemcpyAsync(dst, src, plane * h->g.nz * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
        return AC_OK;
    }
    size_t np;
    int rc = ensure_stage(h, &np);
    if (rc) return rc;
    for (size_t z0 = 0; z0 < (size_t)h->g.nz; z0 += np) {
        const size_t nzc = (z0 + np <= (size_t)h->g.nz) ? np : (size_t)h->g.nz - z0;
        CK(launch_gather(src, es, h->g, (int)z0, (int)nzc, h->stage, h->stream));
        h->launches++;
        CK(cudaMemcpyAsync(dst + z0 * plane, h->stage, nzc * plane * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    }
    return AC_OK;
}

static int load_common(ac_handle *h, int field, const double *src, int to_w) {
    if (!h || !src || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    int rc = ensure_state(h);
    if (rc) return rc;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    for (int q = q0; q < q1; ++q) {
        const double *s = src + (field == AC_ALL ? (size_t)q * n : 0);
        rc = to_w ? load_array(h, h->w[q], h->elem_w, s)
                  : load_array(h, h->state[h->cur][q], h->elem_f, s);
        if (rc) return rc;
    }
    if (!to_w) h->next_s = 0;
    return AC_OK;
}

static int store_common(ac_handle *h, int field, double *dst, int from_w) {
    if (!h || !dst || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    int rc = ensure_state(h);
    if (rc) return rc;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    for (int q = q0; q < q1; ++q) {
        double *d = dst + (field == AC_ALL ? (size_t)q * n : 0);
        rc = from_w ? store_array(h, h->w[q], h->elem_w, d)
                    : store_array(h, h->state[h->cur][q], h->elem_f, d);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return AC_OK;
}

// Host binary32 format: the state's own bytes when it is binary32 in the periodic
// layout, else through the staging buffer (binary32 values, twice the planes).
static int load_array_f32(ac_handle *h, void *dst, int es, const float *src) {
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    if (es == 4 && !h->g.padded) {
        CK(cudaMemcpyAsync(dst, src, plane * h->g.nz * sizeof(float), cudaMemcpyHostToDevice,
                           h->stream));
        return AC_OK;
    }
    size_t np;
    int rc = ensure_stage(h, &np);
    if (rc) return rc;
    np *= 2;  // the stage holds binary64 planes
    float *stage = reinterpret_cast<float *>(h->stage);
    for (size_t z0 = 0; z0 < (size_t)h->g.nz; z0 += np) {
        const size_t nzc = (z0 + np <= (size_t)h->g.nz) ? np : (size_t)h->g.nz - z0;
        CK(cudaMemcpyAsync(stage, src + z0 * plane, nzc * plane * sizeof(float),
                           cudaMemcpyHostToDevice, h->stream));
        CK(launch_scatter_f32(stage, dst, es, h->g, (int)z0, (int)nzc, h->stream));
        h->launches++;
    }
    return AC_OK;
}

static int store_array_f32(ac_handle *h, const void *src, int es, float *dst) {
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    if (es == 4 && !h->g.padded) {
        CK(cudaMemcpyAsync(dst, src, plane * h->g.nz * sizeof(float), cudaMemcpyDeviceToHost,
                           h->stream));
        return AC_OK;
    }
    size_t np;
    int rc = ensure_stage(h, &np);
    if (rc) return rc;
    np *= 2;
    float *stage = reinterpret_cast<float *>(h->stage);
    for (size_t z0 = 0; z0 < (size_t)h->g.nz; z0 += np) {
        const size_t nzc = (z0 + np <= (size_t)h->g.nz) ? np : (size_t)h->g.nz - z0;
        CK(launch_gather_f32(src, es, h->g, (int)z0, (int)nzc, stage, h->stream));
        h->launches++;
        CK(cudaMemcpyAsync(dst + z0 * plane, stage, nzc * plane * sizeof(float),
                           cudaMemcpyDeviceToHost, h->stream));
    }
    return AC_OK;
}

extern "C" int ac_load_f32(ac_handle *h, int field, const float *src) {
    AC_RANGE("ac_load_f32");
    if (!h || !src || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    int rc = ensure_state(h);
    if (rc) return rc;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    for (int q = q0; q < q1; ++q) {
        rc = load_array_f32(h, h->state[h->cur][q], h->elem_f, src + (field == AC_ALL ? (size_t)q * n : 0));
        if (rc) return rc;
    }
    h->next_s = 0;
    return AC_OK;
}

extern "C" int ac_store_f32(ac_handle *h, int field, float *dst) {
    AC_RANGE("ac_store_f32");
    if (!h || !dst || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    int rc = ensure_state(h);
    if (rc) return rc;
    const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    for (int q = q0; q < q1; ++q) {
        rc = store_array_f32(h, h->state[h->cur][q], h->elem_f, dst + (field == AC_ALL ? (size_t)q * n : 0));
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return AC_OK;
}

extern "C" int ac_load(ac_handle *h, int field, const double *src) {
    AC_RANGE("ac_load");
    return load_common(h, field, src, 0);
}
extern "C" int ac_store(ac_handle *h, int field, double *dst) {
    AC_RANGE("ac_store");
    return store_common(h, field, dst, 0);
}
extern "C" int ac_load_w(ac_handle *h, int field, const double *src) {
    return load_common(h, field, src, 1);
}
extern "C" int ac_store_w(ac_handle *h, int field, double *dst) {
    return store_common(h, field, dst, 1);
}

extern "C" int ac_periodic_halo(ac_handle *h) {
    if (!h) return AC_ERR_ARG;
    if (!h->g.padded) return AC_OK;
    int rc = ensure_state(h);
    if (rc) return rc;
    CK(launch_halo(h->params.precision, h->g, h->state[h->cur], h->stream));
    h->launches++;
    return AC_OK;
}

// ---- forcing --------------------------------------------------------------

static uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    // SplitMix64 (Steele, Lea, Flood 2014): n-th output of the stream seeded with `seed`.
    uint64_t z = seed + (counter + 1u) * UINT64_C(0x9E3779B97F4A7C15);
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

static double unit_double(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

extern "C" int ac_forcing_draw(unsigned long long seed, unsigned long long step, int k[3],
                               double e[3], double *phi) {
    if (!k || !e || !phi) return AC_ERR_ARG;
    // The shell 4 <= |k|^2 <= 9, enumerated with kx, ky, kz ascending from -3 to 3.
    int shell[343][3];
    int count = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                const int k2 = a * a + b * b + c * c;
                if (k2 >= 4 && k2 <= 9) {
                    shell[count][0] = a;
                    shell[count][1] = b;
                    shell[count][2] = c;
                    ++count;
                }
            }
    const uint64_t base = 16ull * step;
    const int pick = (int)(splitmix64(seed, base) % (uint64_t)count);
    const int ki[3] = {shell[pick][0], shell[pick][1], shell[pick][2]};
    const double kk[3] = {(double)ki[0], (double)ki[1], (double)ki[2]};
    const double k2 = kk[0] * kk[0] + kk[1] * kk[1] + kk[2] * kk[2];
    // A helper vector not parallel to k: up to four uniform draws in the cube, else an axis.
    double v[3] = {0.0, 0.0, 0.0};
    int ok = 0;
    for (int t = 0; t < 4 && !ok; ++t) {
        double c[3];
        for (int a = 0; a < 3; ++a)
            c[a] = 2.0 * unit_double(splitmix64(seed, base + 1 + 3 * t + a)) - 1.0;
        const double x0 = kk[1] * c[2] - kk[2] * c[1];
        const double x1 = kk[2] * c[0] - kk[0] * c[2];
        const double x2 = kk[0] * c[1] - kk[1] * c[0];
        const double xx = x0 * x0 + x1 * x1 + x2 * x2;
        const double cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        if (cc >= 1.0 / 16.0 && xx >= 0.25 * k2 * cc) {
            v[0] = c[0];
            v[1] = c[1];
            v[2] = c[2];
            ok = 1;
        }
    }
    if (!ok) {
        int best = 0;
        for (int a = 1; a < 3; ++a)
            if (abs(ki[a]) < abs(ki[best])) best = a;
        v[best] = 1.0;
    }
    const double p0 = kk[1] * v[2] - kk[2] * v[1];
    const double p1 = kk[2] * v[0] - kk[0] * v[2];
    const double p2 = kk[0] * v[1] - kk[1] * v[0];
    const double pn = sqrt(p0 * p0 + p1 * p1 + p2 * p2);
    k[0] = ki[0];
    k[1] = ki[1];
    k[2] = ki[2];
    e[0] = p0 / pn;
    e[1] = p1 / pn;
    e[2] = p2 / pn;
    *phi = 6.283185307179586476925286766559 * unit_double(splitmix64(seed, base + 13));
    return AC_OK;
}

extern "C" int ac_set_forcing(ac_handle *h, const int k[3], const double e[3], double phi) {
    if (!h) return AC_ERR_ARG;
    if (!k) {
        h->force_manual = 0;
        h->ftab_valid = 0;
        return AC_OK;
    }
    if (!e || !isfinite(phi) || !isfinite(e[0]) || !isfinite(e[1]) || !isfinite(e[2]))
        return AC_ERR_ARG;
    h->force_manual = 1;
    for (int a = 0; a < 3; ++a) {
        h->force_k[a] = k[a];
        h->force_e[a] = e[a];
    }
    h->force_phi = phi;
    h->ftab_dirty = 1;
    h->ftab_valid = 0;
    return AC_OK;
}

// Integer stencil sums apply to binary64 fields on a periodic grid with equal
// spacing on every axis (so numerators of different axes share a coefficient).
static int fx_applicable(const ac_handle *h) {
    const double dx = h->grid.lx / h->grid.nx, dy = h->grid.ly / h->grid.ny,
                 dz = h->grid.lz / h->grid.nz;
    return h->params.precision == AC_FP64 && h->grid.layout == AC_LAYOUT_PERIODIC && dx == dy &&
           dy == dz && h->coefs.radius == 3;
}

extern "C" int ac_set_stencil_mode(ac_handle *h, int mode) {
    if (!h || mode < AC_STENCIL_AUTO || mode > AC_STENCIL_FIXED) return AC_ERR_ARG;
    if (mode == AC_STENCIL_FIXED && !fx_applicable(h)) return AC_ERR_ARG;
    h->stencil_mode = mode;
    return AC_OK;
}

extern "C" int ac_set_entropy_terms(ac_handle *h, double K, double zeta, double heat,
                                    double cool) {
    if (!h || !isfinite(K) || !isfinite(zeta) || !isfinite(heat) || !isfinite(cool) || K < 0.0 ||
        zeta < 0.0 || heat < 0.0 || cool < 0.0)
        return AC_ERR_ARG;
    h->phys.K = K;
    h->phys.zeta = zeta;
    h->phys.hc = heat - cool;
    return AC_OK;
}

extern "C" int ac_set_stencil_order(ac_handle *h, int order) {
    if (!h || (order != 2 && order != 4 && order != 6 && order != 8)) return AC_ERR_ARG;
    if (h->grid.layout == AC_LAYOUT_PADDED && order > 6) return AC_ERR_ARG;  // halo is 3 wide
    if (h->next_s != 0) return AC_ERR_STATE;  // only at a step boundary
    const int old = h->coefs.radius;
    const double dx[3] = {h->grid.lx / h->grid.nx, h->grid.ly / h->grid.ny, h->grid.lz / h->grid.nz};
    h->coefs = make_coefs(dx, order / 2);
    if (h->stencil_mode == AC_STENCIL_FIXED && !fx_applicable(h)) {
        h->coefs = make_coefs(dx, old);
        return AC_ERR_ARG;
    }
    return AC_OK;
}

extern "C" int ac_get_stencil_order(const ac_handle *h, int *order) {
    if (!h || !order) return AC_ERR_ARG;
    *order = 2 * h->coefs.radius;
    return AC_OK;
}

extern "C" int ac_get_stencil_path(const ac_handle *h, int *fixed) {
    if (!h || !fixed) return AC_ERR_ARG;
    *fixed = h->stencil_mode != AC_STENCIL_FP64 && fx_applicable(h);
    return AC_OK;
}

// Elements between the int64 copies of consecutive fields: even, so that every
// copy starts on a 16-byte boundary (the quantisation stores two at a time).
static size_t fx_stride(const ac_handle *h) { return ((size_t)h->g.elems + 1) & ~(size_t)1; }

// Work areas of the integer-sum path, on first use: the int64 copies of the
// fields, the extremes words and the plan (zeroed, so its mode counts start at 0).
static int ensure_fx(ac_handle *h) {
    if (h->fx_block) return AC_OK;
    long long *blk = nullptr;
    unsigned long long *stats = nullptr;
    void *plan = nullptr;
    cudaError_t e = cudaMalloc(&blk, (size_t)NF * fx_stride(h) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&stats, 2 * NF * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&plan, fx_plan_bytes());
    if (e == cudaSuccess) e = cudaMemsetAsync(plan, 0, fx_plan_bytes(), h->stream);
    // extremes: largest keys start at 0, smallest at all ones (the plan kernel
    // restores this after every read)
    if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, NF * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(stats + NF, 0xff, NF * sizeof(unsigned long long), h->stream);
    if (e != cudaSuccess) {
        if (blk) cudaFree(blk);
        if (stats) cudaFree(stats);
        if (plan) cudaFree(plan);
        return cuda_fail(e);
    }
    h->fx_block = blk;
    h->fx_stats = stats;
    h->fx_plan = plan;
    return AC_OK;
}

extern "C" int ac_get_stencil_modes(ac_handle *h, unsigned long long counts[3]) {
    if (!h || !counts) return AC_ERR_ARG;
    counts[0] = counts[1] = counts[2] = 0;
    if (!h->fx_plan) return AC_OK;
    CK(fx_plan_taken(h->fx_plan, counts, h->stream));
    return AC_OK;
}

extern "C" int ac_get_step(const ac_handle *h, unsigned long long *step, int *next_substep) {
    if (!h) return AC_ERR_ARG;
    if (step) *step = h->step;
    if (next_substep) *next_substep = h->next_s;
    return AC_OK;
}

extern "C" int ac_set_step(ac_handle *h, unsigned long long step, int next_substep) {
    if (!h || next_substep < 0 || next_substep > 2) return AC_ERR_ARG;
    h->step = step;
    h->next_s = next_substep;
    return AC_OK;
}

extern "C" int ac_get_state(const ac_handle *h, void *dev_ptrs[8], int *precision, int *layout,
                            int n[3]) {
    if (!h) return AC_ERR_ARG;
    if (dev_ptrs) {
        if (!h->have_buffers) return AC_ERR_STATE;
        for (int q = 0; q < NF; ++q) dev_ptrs[q] = h->state[h->cur][q];
    }
    if (precision) *precision = h->params.precision;
    if (layout) *layout = h->grid.layout;
    if (n) {
        n[0] = h->grid.nx;
        n[1] = h->grid.ny;
        n[2] = h->grid.nz;
    }
    return AC_OK;
}

extern "C" int ac_launch_count(const ac_handle *h, unsigned long long *count) {
    if (!h || !count) return AC_ERR_ARG;
    *count = h->launches;
    return AC_OK;
}

// ---- integration ------------------------------------------------------------

#ifdef AC_BOUNDS_CHECK
namespace ac {
unsigned long long bc_take_aux();
unsigned long long bc_take_batch();
unsigned long long bc_take_closure();
unsigned long long bc_take_decomp();
unsigned long long bc_take_noalloc();
unsigned long long bc_take_f32();
unsigned long long bc_take_f32g();
unsigned long long bc_take_f64();
}  // namespace ac
#endif

extern "C" int ac_bounds_check_take(unsigned long long *first) {
    if (!first) return AC_ERR_ARG;
    *first = 0;
#ifdef AC_BOUNDS_CHECK
    unsigned long long (*const readers[])() = {bc_take_aux,     bc_take_batch, bc_take_closure,
                                               bc_take_decomp,  bc_take_noalloc, bc_take_f32,
                                               bc_take_f32g,    bc_take_f64};
    for (auto r : readers) {
        const unsigned long long w = r();
        if (w == ~0ull) return AC_ERR_CUDA;
        if (!*first) *first = w;
    }
    return AC_OK;
#else
    return AC_ERR_STATE;  // the library was compiled without the index checks
#endif
}

extern "C" int ac_integrate_substep(ac_handle *h, double dt, int s) {
    AC_RANGE("ac_integrate_substep");
    if (!h || s < 0 || s > 2 || !isfinite(dt)) return AC_ERR_ARG;
    if (s != h->next_s) return AC_ERR_STATE;
    int rc = ensure_state(h);
    if (rc) return rc;
    const int forcing = h->params.force_amp != 0.0;
    if (forcing) {
        // Per-step draw: (k, e, phi) stay fixed over the three substeps of a step.
        if (!h->force_manual && (!h->ftab_valid || h->ftab_step != h->step)) {
            ac_forcing_draw(h->params.seed, h->step, h->force_k, h->force_e, &h->force_phi);
            h->ftab_step = h->step;
            h->ftab_dirty = 1;
        }
        if (h->ftab_dirty || !h->ftab_valid) {
            CK(launch_forcing_table(h->g, h->force_k, h->force_phi, h->ftab, h->stream));
            h->launches++;
            h->ftab_dirty = 0;
            h->ftab_valid = 1;
        }
    }
    if (h->g.padded) {
        CK(launch_halo(h->params.precision, h->g, h->state[h->cur], h->stream));
        h->launches++;
    }
    SubstepLaunch L;
    L.precision = h->params.precision;
    L.g = h->g;
    for (int q = 0; q < NF; ++q) {
        L.fin[q] = h->state[h->cur][q];
        L.fout[q] = h->state[1 - h->cur][q];
        L.w[q] = h->w[q];
    }
    L.c = h->coefs;
    L.ph = h->phys;
    L.force.on = forcing;
    L.force.tab = h->ftab;
    for (int a = 0; a < 3; ++a) L.force.amp_e[a] = h->params.force_amp * h->force_e[a];
    L.alpha = RK_ALPHA[s];
    L.beta = RK_BETA[s];
    L.dt = dt;
    L.s = s;
    // (integer sums need 32-bit neighbour offsets: fewer than 2^31 cells per array)
    L.use_fx = h->stencil_mode != AC_STENCIL_FP64 && fx_applicable(h) &&
               h->g.elems < (1ll << 31);
    L.dx = h->grid.lx / h->grid.nx;
    L.fx_stats = nullptr;
    L.fx_plan = nullptr;
    for (int q = 0; q < NF; ++q) L.fxF[q] = nullptr;
    if (L.use_fx) {
        rc = ensure_fx(h);
        if (rc) return rc;
        for (int q = 0; q < NF; ++q) L.fxF[q] = h->fx_block + (size_t)q * fx_stride(h);
        L.fx_stats = h->fx_stats;
        L.fx_plan = h->fx_plan;
    }
    L.ev_mid = nullptr;
    cudaEvent_t *tev = nullptr;
    if (h->timing && h->nrec < AC_TIMING_MAX) {
        tev = h->tev + 3 * h->nrec;
        h->trec_s[h->nrec++] = s;
        CK(cudaEventRecord(tev[0], h->stream));
        if (L.use_fx)
            L.ev_mid = tev[1];  // recorded by the launcher after its preparation kernels
        else
            CK(cudaEventRecord(tev[1], h->stream));  // no preparation kernels
    }
    L.cfl_max = nullptr;
    if (s == 0) {  // the step's input state: record its max CFL speed on the way
        CK(cudaMemsetAsync(h->cfl_dev, 0, sizeof(unsigned long long), h->stream));
        L.cfl_max = h->cfl_dev;
    }
    int nl = 0;
    cudaError_t e;
    if (h->params.precision == AC_FP64)
        e = launch_substep_f64(L, h->stream, &nl);
    else if (h->params.precision == AC_FP32)
        e = launch_substep_f32(L, h->stream, &nl);
    else
        e = launch_substep_f32w64(L, h->stream, &nl);
    h->launches += nl;
    if (e != cudaSuccess) return cuda_fail(e);
    if (tev) CK(cudaEventRecord(tev[2], h->stream));
    h->cur = 1 - h->cur;
    h->next_s = (s + 1) % 3;
    if (s == 2) h->step++;
    return AC_OK;
}

extern "C" int ac_set_kernel_timing(ac_handle *h, int on) {
    if (!h) return AC_ERR_ARG;
    if (on && !h->tev) {
        h->tev = static_cast<cudaEvent_t *>(calloc(3 * AC_TIMING_MAX, sizeof(cudaEvent_t)));
        if (!h->tev) return AC_ERR_OOM;
        for (int i = 0; i < 3 * AC_TIMING_MAX; ++i) {
            cudaError_t e = cudaEventCreate(&h->tev[i]);
            if (e != cudaSuccess) {
                free_timing(h);
                return cuda_fail(e);
            }
        }
    }
    h->timing = on != 0;
    h->nrec = 0;
    return AC_OK;
}

extern "C" int ac_kernel_timings(ac_handle *h, double prep_ms[3], double kernel_ms[3],
                                 int count[3]) {
    if (!h || !prep_ms || !kernel_ms || !count) return AC_ERR_ARG;
    for (int s = 0; s < 3; ++s) {
        prep_ms[s] = kernel_ms[s] = 0.0;
        count[s] = 0;
    }
    if (h->nrec) CK(cudaEventSynchronize(h->tev[3 * (h->nrec - 1) + 2]));
    for (int r = 0; r < h->nrec; ++r) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, h->tev[3 * r], h->tev[3 * r + 1]));
        CK(cudaEventElapsedTime(&b, h->tev[3 * r + 1], h->tev[3 * r + 2]));
        const int s = h->trec_s[r];
        prep_ms[s] += a;
        kernel_ms[s] += b;
        count[s]++;
    }
    for (int s = 0; s < 3; ++s)
        if (count[s]) {
            prep_ms[s] /= count[s];
            kernel_ms[s] /= count[s];
        }
    h->nrec = 0;
    return AC_OK;
}

extern "C" int ac_integrate_step(ac_handle *h, double dt) {
    AC_RANGE("ac_integrate_step");
    if (!h || !isfinite(dt)) return AC_ERR_ARG;
    if (h->next_s != 0) return AC_ERR_STATE;
    for (int s = 0; s < 3; ++s) {
        int rc = ac_integrate_substep(h, dt, s);
        if (rc) return rc;
    }
    return AC_OK;
}

extern "C" int ac_last_cfl(ac_handle *h, double *out) {
    if (!h || !out) return AC_ERR_ARG;
    CK(cudaMemcpyAsync(h->result_host, h->cfl_dev, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *out = h->result_host[0];
    return isfinite(*out) ? AC_OK : AC_ERR_NONFINITE;
}

// ---- reductions -------------------------------------------------------------

extern "C" int ac_reduce(ac_handle *h, int op, int quantity, double *out) {
    AC_RANGE("ac_reduce");
    if (!h || !out || op < AC_MAX || op > AC_RMS || quantity < 0 || quantity > AC_Q_CFL)
        return AC_ERR_ARG;
    int rc = ensure_state(h);
    if (rc) return rc;
    if (h->g.padded) {  // derived quantities read neighbours through the halo
        CK(launch_halo(h->params.precision, h->g, h->state[h->cur], h->stream));
        h->launches++;
    }
    ReduceLaunch L;
    L.precision = h->params.precision;
    L.g = h->g;
    for (int q = 0; q < NF; ++q) L.f[q] = h->state[h->cur][q];
    L.c = h->coefs;
    L.ph = h->phys;
    L.op = op;
    L.quantity = quantity;
    L.partials = h->partials;
    L.flags = h->flags;
    L.result = h->result_dev;
    L.blocks = reduce_max_blocks();
    int nl = 0;
    cudaError_t e = launch_reduce(L, h->stream, &nl);
    h->launches += nl;
    if (e != cudaSuccess) return cuda_fail(e);
    CK(cudaMemcpyAsync(h->result_host, h->result_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *out = h->result_host[0];
    unsigned int flag;
    memcpy(&flag, &h->result_host[1], sizeof flag);
    return flag ? AC_ERR_NONFINITE : AC_OK;
}
