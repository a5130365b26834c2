// Binary32 substep kernels: the shared-memory tiled z-marching kernel for the
// periodic layout at the sixth order of Sec. 4, the direct-load kernel for the
// padded layout and for the other stencil orders.
#include "substep_tiled.cuh"

namespace ac {
cudaError_t launch_substep_f32(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    if (!L.g.padded && L.c.radius == 3) return launch_substep_tiled_t<float>(L, st, launches);
    return launch_substep_t<float, float>(L, st, launches);
}
cudaError_t launch_substep_f32w64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    if (!L.g.padded && L.c.radius == 3) return launch_substep_tiled_t<double>(L, st, launches);
    return launch_substep_t<float, double>(L, st, launches);
}
}  // namespace ac
