// op_min_f32.cu -- forward passes with the minimum along the patterns over
// float32 images and levels.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_min_f32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, float, float, float, float, 2>(M, d, st);
}
}  // namespace fht
