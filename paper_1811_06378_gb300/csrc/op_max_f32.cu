// op_max_f32.cu -- forward passes with the maximum along the patterns over
// float32 images and levels.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_max_f32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, float, float, float, float, 1>(M, d, st);
}
}  // namespace fht
