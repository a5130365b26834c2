// Binary32 substep kernels: the shared-memory tiled z-marching kernel for the
// periodic layout at the sixth order of Sec. 4; the direct-load kernel (padded
// layout, other stencil orders) is compiled separately in k_substep_f32g.cu.
#include "substep_tiled.cuh"

namespace ac {
cudaError_t launch_substep_f32_direct(const SubstepLaunch &L, cudaStream_t st, int *launches,
                                      bool w64);

cudaError_t launch_substep_f32(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    if (!L.g.padded && L.c.radius == 3) return launch_substep_tiled_t<float>(L, st, launches);
    return launch_substep_f32_direct(L, st, launches, false);
}
cudaError_t launch_substep_f32w64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    if (!L.g.padded && L.c.radius == 3) return launch_substep_tiled_t<double>(L, st, launches);
    return launch_substep_f32_direct(L, st, launches, true);
}
}  // namespace ac

AC_BC_READER(bc_take_f32)
