// fused_f32_u8.cu -- fused forward pass instantiations: accumulator float,
// source uint8_t, shared tile float, destination float.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_fused_f32_u8(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, float, uint8_t, float, float>(M, d, st);
}
}  // namespace fht
