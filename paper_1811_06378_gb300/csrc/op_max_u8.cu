// op_max_u8.cu -- forward passes with the maximum along the patterns in place
// of the sum, over uint8 images: first passes into a uint16 level, and
// single passes straight to int32.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_max_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, int32_t, uint8_t, uint16_t, uint16_t, 1>(M, d, st);
}
cudaError_t launch_max_i32_u8_i32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, int32_t, uint8_t, uint16_t, int32_t, 1>(M, d, st);
}
}  // namespace fht
