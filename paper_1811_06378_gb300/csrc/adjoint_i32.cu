// adjoint_i32.cu -- adjoint pass instantiations (opposite-sign cyclic
// transform of a int32_t gradient into the image gradient).
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_i32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, int32_t, int32_t, int32_t, int32_t>(M, d, st);
}
}  // namespace fht
