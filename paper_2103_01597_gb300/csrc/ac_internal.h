// Internal declarations shared by the C-ABI implementation and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "ac.h"

namespace ac {

// An NVTX range named after the C call for its whole extent (shows in profiler
// timelines; costs a call into the NVTX stub when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define AC_RANGE(name) ::ac::NvtxRange ac_nvtx_range_(name)


constexpr int NF = 8;
constexpr int R = 3;  // stencil radius (sixth order, Sec. 4)

// Geometry of one device field array.  Periodic layout: px = nx, pxy = nx*ny,
// origin 0.  Padded layout: px = nx + 6, pxy = px * (ny + 6) and the interior
// origin is 3 * (1 + px + pxy).
struct Geom {
    int nx, ny, nz;
    int padded;
    int px;
    long long pxy;
    long long origin;
    long long elems;  // elements per array
};

inline Geom make_geom(int nx, int ny, int nz, int layout) {
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.padded = layout == AC_LAYOUT_PADDED;
    if (g.padded) {
        g.px = nx + 2 * R;
        g.pxy = (long long)g.px * (ny + 2 * R);
        g.origin = R * (1 + g.px + g.pxy);
        g.elems = g.pxy * (nz + 2 * R);
    } else {
        g.px = nx;
        g.pxy = (long long)nx * ny;
        g.origin = 0;
        g.elems = g.pxy * nz;
    }
    return g;
}

// Stencil coefficients with the grid spacing folded in (host side, binary64),
// for central differences of order 2r, radius r = 1 .. 4 (r = 3 is Sec. 4's).
constexpr int MAX_RADIUS = 4;
struct StencilCoefs {
    double d1[3][MAX_RADIUS];      // first derivative: [axis][m-1] multiplies (f_m - f_-m)
    double d2[3][MAX_RADIUS + 1];  // second derivative: [axis][0] centre, [axis][m] (f_m + f_-m)
    double dc[3][MAX_RADIUS];      // mixed: plane 0 = xy, 1 = xz, 2 = yz; [m-1] multiplies S_m
    int radius;
};
StencilCoefs make_coefs(const double dx[3], int radius = 3);

// Physical constants of Eqs. B.1-B.4 in the form the kernels use.
struct PhysConsts {
    double nu, eta;
    double inv_cp;      // 1 / c_p
    double cs2_ref;     // c_s0^2 exp(-(gamma - 1) lnrho0)
    double gamma_cp;    // gamma / c_p
    double gm1;         // gamma - 1
    double cp_gm1;      // c_p (gamma - 1): 1/T = c_p (gamma - 1) / c_s^2
    // Eq. B.2-B.3 terms beyond the base configuration (all 0 by default):
    double K;           // thermal conductivity
    double zeta;        // bulk viscosity
    double hc;          // heating minus cooling, H - C
    bool ext() const { return K != 0.0 || zeta != 0.0 || hc != 0.0; }
};
PhysConsts make_phys(const ac_params &p);

// Forcing of the current step, device tables of e^{i theta_a(i)}.
struct ForceArgs {
    int on;
    const double2 *tab;  // [nx] then [ny] then [nz] entries; the z table includes phi
    double amp_e[3];     // force_amp * e
};

struct SubstepLaunch {
    int precision;
    Geom g;
    const void *fin[NF];
    void *fout[NF];
    void *w[NF];
    StencilCoefs c;
    PhysConsts ph;
    ForceArgs force;
    double alpha, beta, dt;
    int s;
    unsigned long long *cfl_max;  // substep 0: device word for the max CFL speed (or NULL)
    // binary64 with integer stencil sums (cubic periodic grids): int64 copies of
    // the fields, 16 words of per-field extremes and the device plan of the
    // substep (fx_plan_bytes()); use_fx = 0 selects plain binary64 sums.
    int use_fx;
    long long *fxF[NF];
    unsigned long long *fx_stats;
    void *fx_plan;
    double dx;
    // optional: recorded after the preparation kernels (integer-sum path:
    // extremes, plan, quantisation), before the substep kernel itself
    cudaEvent_t ev_mid;
};
size_t fx_plan_bytes();
// Substeps run in each mode (group scales, per-field scales, plain binary64)
// since the plan was zeroed; synchronises `st`.
cudaError_t fx_plan_taken(const void *plan, unsigned long long taken[3], cudaStream_t st);

cudaError_t launch_substep(const SubstepLaunch &L, cudaStream_t st, int *launches);
cudaError_t launch_halo(int precision, const Geom &g, void *const f[NF], cudaStream_t st);
cudaError_t launch_forcing_table(const Geom &g, const int k[3], double phi, double2 *tab,
                                 cudaStream_t st);
// Convert/scatter one z-slab of an unpadded float64 staging buffer into a
// device array of the given element size (4 or 8), and back.
cudaError_t launch_scatter(const double *stage, void *dst, int elem_size, const Geom &g, int z0,
                           int nzc, cudaStream_t st);
cudaError_t launch_gather(const void *src, int elem_size, const Geom &g, int z0, int nzc,
                          double *stage, cudaStream_t st);
// The same with a binary32 staging buffer (host binary32 format).
cudaError_t launch_scatter_f32(const float *stage, void *dst, int elem_size, const Geom &g, int z0,
                               int nzc, cudaStream_t st);
cudaError_t launch_gather_f32(const void *src, int elem_size, const Geom &g, int z0, int nzc,
                              float *stage, cudaStream_t st);

struct ReduceLaunch {
    int precision;
    Geom g;
    const void *f[NF];
    StencilCoefs c;
    PhysConsts ph;
    int op, quantity;
    double *partials;      // scratch, >= reduce_max_blocks() doubles
    unsigned int *flags;   // scratch, >= reduce_max_blocks() words (non-finite seen)
    double *result;        // one double + one flag word after it (device)
    int blocks;
};
int reduce_max_blocks();
cudaError_t launch_reduce(const ReduceLaunch &L, cudaStream_t st, int *launches);

// Record a CUDA error for ac_last_cuda_error() and map it to an AC_ERR_* code.
int ac_report_cuda(cudaError_t e);

// Argument checks of ac_init: 1 if the grid (positive finite box lengths, a
// known layout, every axis at most 2^24 cells) or the parameters (finite,
// nu, eta >= 0, c_s0, c_p > 0, gamma > 1, a known precision) are valid.
int valid_grid(const ac_grid *g);
int valid_params(const ac_params *p);

}  // namespace ac
