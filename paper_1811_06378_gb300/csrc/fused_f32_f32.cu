// fused_f32_f32.cu -- fused forward pass instantiations: accumulator float,
// source float, shared tile float, destination float.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_fused_f32_f32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, float, float, float, float>(M, d, st);
}
}  // namespace fht
