// FP64 substep: exact integer stencil sums on cubic periodic grids (the fast
// path), plain binary64 stencil arithmetic otherwise.
#include "substep_fx.cuh"

namespace ac {

static unsigned fx_grid(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

cudaError_t launch_substep_f64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    if (!L.use_fx) return launch_substep_t<double, double>(L, st, launches);
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
    FxCoefs fc;
    fc.inv60dx = 1.0 / (60.0 * L.dx);
    fc.nu180 = L.ph.nu / (180.0 * L.dx * L.dx);
    fc.nu2160 = (L.ph.nu + 3.0 * L.ph.zeta) / (2160.0 * L.dx * L.dx);
    fc.inv180dx2 = 1.0 / (180.0 * L.dx * L.dx);
    fc.inv720dx2 = 1.0 / (720.0 * L.dx * L.dx);

    const long long n = L.g.elems;
    cudaError_t e = cudaMemsetAsync(L.fx_gmax, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    fx_max_kernel<<<fx_grid(n), 256, 0, st>>>(fx, n, L.fx_gmax);
    fx_quantize_kernel<<<fx_grid(n), 256, 0, st>>>(fx, n, L.fx_gmax);

    const dim3 block(32, 4, 1);
    const unsigned gx = (L.g.nx + block.x - 1) / block.x;
    const unsigned gy = (L.g.ny + block.y - 1) / block.y;
    const long long xy_blocks = (long long)gx * gy;
    int zchunk = (int)((xy_blocks * L.g.nz) / (8 * 152));
    zchunk = zchunk < 1 ? 1 : (zchunk > 16 ? 16 : zchunk);
    a.zchunk = zchunk;
    const dim3 grid(gx, gy, (L.g.nz + zchunk - 1) / zchunk);
    // 32-bit neighbour offsets whenever they fit (always, for binary64 state in
    // 280 GB: fewer than 2^31 cells), 64-bit otherwise
    const bool off32 = L.g.elems < (1ll << 31);
    const bool ext = L.ph.ext(), cfl = a.cfl_max != nullptr;
#define AC_FX(IX, C, X) substep_fx_kernel<IX, C, X><<<grid, block, 0, st>>>(a, fx, fc, L.fx_gmax)
    if (off32) {
        if (ext) { if (cfl) AC_FX(IdxPeriodic32, true, true); else AC_FX(IdxPeriodic32, false, true); }
        else { if (cfl) AC_FX(IdxPeriodic32, true, false); else AC_FX(IdxPeriodic32, false, false); }
    } else {
        if (ext) { if (cfl) AC_FX(IdxPeriodic, true, true); else AC_FX(IdxPeriodic, false, true); }
        else { if (cfl) AC_FX(IdxPeriodic, true, false); else AC_FX(IdxPeriodic, false, false); }
    }
#undef AC_FX
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace ac

AC_BC_READER(bc_take_f64)
