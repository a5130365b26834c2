// FP32 instantiations of the fused substep kernel (binary32 or binary64 accumulator).
#include "substep.cuh"

namespace ac {
cudaError_t launch_substep_f32(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    return launch_substep_t<float, float>(L, st, launches);
}
cudaError_t launch_substep_f32w64(const SubstepLaunch &L, cudaStream_t st, int *launches) {
    return launch_substep_t<float, double>(L, st, launches);
}
}  // namespace ac
