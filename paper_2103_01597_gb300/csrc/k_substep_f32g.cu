// Binary32 substep on the direct-load kernel (global-memory stencil loads):
// the padded layout and the stencil orders other than six.
#include "substep.cuh"

namespace ac {
cudaError_t launch_substep_f32_direct(const SubstepLaunch &L, cudaStream_t st, int *launches,
                                      bool w64) {
    return w64 ? launch_substep_t<float, double>(L, st, launches)
               : launch_substep_t<float, float>(L, st, launches);
}
}  // namespace ac

AC_BC_READER(bc_take_f32g)
