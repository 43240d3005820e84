// fused_i32_i32.cu -- fused forward pass instantiations: accumulator int32_t,
// source int32_t, shared tile int32_t, destination int32_t.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_fused_i32_i32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, int32_t, int32_t, int32_t, int32_t>(M, d, st);
}
}  // namespace fht
