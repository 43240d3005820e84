// sheared_i32_u8_u16.cu -- cyclic pass instantiations of the sheared forward
// transform (Section 4): first passes over uint8 images into a uint16 level
// (accumulator int32_t, source uint8_t, shared tile uint16_t, destination uint16_t).
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, int32_t, uint8_t, uint16_t, uint16_t>(M, d, st);
}
}  // namespace fht
