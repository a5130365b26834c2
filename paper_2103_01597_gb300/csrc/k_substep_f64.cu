// FP64 instantiation of the fused substep kernel.
#include "substep.cuh"

namespace ac {
cudaError_t launch_substep_f64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    return launch_substep_t<double, double>(L, st, launches);
}
}  // namespace ac
