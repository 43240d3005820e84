// sheared_i32_u16.cu -- cyclic pass instantiations of the sheared forward
// transform (Section 4): passes that read a uint16 level
// (accumulator int32_t, source uint16_t, shared tile int32_t, destination int32_t).
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_i32_u16(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, int32_t, uint16_t, int32_t, int32_t>(M, d, st);
}
}  // namespace fht
