// FP64 substep: exact integer stencil sums on cubic periodic grids (the fast
// path), plain binary64 stencil arithmetic otherwise.
#include <cmath>

#include "substep_fx.cuh"

namespace ac {

static unsigned fx_grid(long long n) {  // n work items of one thread each
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

cudaError_t launch_substep_f64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    // Integer sums need 32-bit neighbour offsets (always true for a binary64
    // state in HBM: fewer than 2^31 cells per array); their kernels fold dt into
    // the coefficients, so a step of zero or of extreme magnitude (1 / dt^2 out of
    // range) takes the plain binary64 stencils.
    const double adt = fabs(L.dt);
    if (!L.use_fx || L.g.elems >= (1ll << 31) || !(adt >= 1e-100 && adt <= 1e100))
        return launch_substep_t<double, double>(L, st, launches);
    SubstepArgs<double, double> a;
    a.g = L.g;
    FxPtrs fx;
    for (int q = 0; q < NF; ++q) {
        a.fin[q] = static_cast<const double *>(L.fin[q]);
        a.fout[q] = static_cast<double *>(L.fout[q]);
        a.w[q] = static_cast<double *>(L.w[q]);
        fx.f[q] = a.fin[q];
        fx.F[q] = L.fxF[q];
    }
    a.k = to_dev<double>(L.c, L.ph);
    a.alpha = L.alpha;
    a.beta = L.beta;
    a.dt = L.dt;
    a.s0 = L.s == 0;
    a.force_on = L.force.on;
    a.ftab = L.force.tab;
    for (int m = 0; m < 3; ++m) a.amp_e[m] = L.force.amp_e[m];
    a.cfl_max = L.cfl_max;
    // the step folded into the RHS coefficients
    FxCoefs fc;
    const double dts = L.dt;
    const double c1 = 1.0 / (60.0 * L.dx);
    fc.c1dt = dts * c1;
    fc.nu180 = dts * (L.ph.nu / (180.0 * L.dx * L.dx));
    fc.nu2160 = dts * ((L.ph.nu + 3.0 * L.ph.zeta) / (2160.0 * L.dx * L.dx));
    fc.inv180dx2 = 1.0 / (180.0 * L.dx * L.dx);
    fc.inv720dx2 = 1.0 / (720.0 * L.dx * L.dx);
    fc.two_nu_c1sq = dts * (2.0 * L.ph.nu * c1 * c1);
    fc.K_c1sq = dts * (L.ph.K * c1 * c1);
    fc.zeta_c1sq = dts * (L.ph.zeta * c1 * c1);
    fc.eta_dt = dts * a.k.eta;
    fc.hc_dt = dts * a.k.hc;
    fc.K_dt = dts * a.k.K;
    for (int m = 0; m < 3; ++m) fc.amp_dt[m] = dts * L.force.amp_e[m];
    fc.inv_dt2 = 1.0 / (dts * dts);

    const long long n = L.g.elems;
    FxPlan *plan = static_cast<FxPlan *>(L.fx_plan);
    cudaError_t e;
    fx_stats_kernel<<<fx_grid(n / 2), 256, 0, st>>>(fx, n, L.fx_stats);
    fx_plan_kernel<<<1, 32, 0, st>>>(L.fx_stats, plan);
    fx_quantize_kernel<<<fx_grid(n / 2), 256, 0, st>>>(fx, n, plan);
    if (L.ev_mid) {
        e = cudaEventRecord(L.ev_mid, st);
        if (e != cudaSuccess) return e;
    }

    const dim3 block(32, 4, 1);
    const unsigned gx = (L.g.nx + block.x - 1) / block.x;
    const unsigned gy = (L.g.ny + block.y - 1) / block.y;
    const long long xy_blocks = (long long)gx * gy;
    int zchunk = (int)((xy_blocks * L.g.nz) / (8 * 152));
    zchunk = zchunk < 1 ? 1 : (zchunk > 16 ? 16 : zchunk);
    a.zchunk = zchunk;
    const dim3 grid(gx, gy, (L.g.nz + zchunk - 1) / zchunk);
    const bool ext = L.ph.ext(), cfl = a.cfl_max != nullptr;
    // one kernel per mode; the two the plan did not choose return at once
#define AC_FX(C, X)                                                            \
    do {                                                                       \
        substep_fx_kernel<false, C, X><<<grid, block, 0, st>>>(a, fx, fc, plan); \
        substep_fx_kernel<true, C, X><<<grid, block, 0, st>>>(a, fx, fc, plan);  \
        substep_fx_plain_kernel<C, X><<<grid, block, 0, st>>>(a, plan);          \
    } while (0)
    if (ext) { if (cfl) AC_FX(true, true); else AC_FX(false, true); }
    else { if (cfl) AC_FX(true, false); else AC_FX(false, false); }
#undef AC_FX
    *launches += 6;
    return cudaGetLastError();
}

// Size of the device plan of the integer-sum path (allocated by the handle).
size_t fx_plan_bytes() { return sizeof(FxPlan); }

// Substeps run in each mode of the integer-sum path, read from a plan.
cudaError_t fx_plan_taken(const void *plan, unsigned long long taken[3], cudaStream_t st) {
    const FxPlan *p = static_cast<const FxPlan *>(plan);
    cudaError_t e = cudaMemcpyAsync(taken, p->taken, 3 * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// The table-driven exp of the binary64 kernels beside CUDA's exp, for tests:
// y[i] = exp_tab(x[i]), y[n + i] = exp(x[i]), y[2n + i] and y[3n + i] = the pair
// exp(x[i]), exp(-x[i]) from exp_tab_pm; where exp_tab_ok(x[i]) fails, the three
// table values are CUDA's (the kernels' fallback).
__global__ void diag_exp_kernel(const double *x, long long n, double *y) {
    __shared__ double tab[512];
    exp_tab_stage(tab);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        double a, b, c;
        if (exp_tab_ok(v)) {
            a = exp_tab(v, tab);
            exp_tab_pm(v, tab, b, c);
        } else {
            a = exp(v);
            b = exp(v);
            c = exp(-v);
        }
        y[i] = a;
        y[n + i] = exp(v);
        y[2 * n + i] = b;
        y[3 * n + i] = c;
    }
}

}  // namespace ac

extern "C" int ac_diag_exp_table(const double *x, long long n, double *y, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return AC_ERR_ARG;
    if (n == 0) return AC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    ac::diag_exp_kernel<<<blocks, 256, 0, st>>>(x, n, y);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? AC_OK : ac::ac_report_cuda(e);
}

AC_BC_READER(bc_take_f64)
