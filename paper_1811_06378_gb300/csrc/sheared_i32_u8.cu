// sheared_i32_u8.cu -- first passes of the sheared forward transform
// (Section 4) over uint8 images: the cyclic pass code with a uint8 source,
// accumulator int32_t.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_i32_u8(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, int32_t, uint8_t, int32_t, int32_t>(M, d, st);
}
}  // namespace fht
