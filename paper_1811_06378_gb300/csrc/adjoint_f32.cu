// adjoint_f32.cu -- adjoint pass instantiations (opposite-sign cyclic
// transform of a float gradient into the image gradient).
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_f32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, float, float, float, float>(M, d, st);
}
}  // namespace fht
