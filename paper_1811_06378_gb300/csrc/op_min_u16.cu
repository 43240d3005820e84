// op_min_u16.cu -- forward passes with the minimum along the patterns that
// read a uint16 level (a uint8 image's values stay below 2^8): into the next
// uint16 level, or the final int32 output (uint16 shared tiles).
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_min_i32_u16_u16(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, int32_t, uint16_t, uint16_t, uint16_t, 2>(M, d, st);
}
cudaError_t launch_min_i32_u16_i32(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<false, int32_t, uint16_t, uint16_t, int32_t, 2>(M, d, st);
}
}  // namespace fht
