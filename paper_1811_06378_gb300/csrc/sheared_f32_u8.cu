// sheared_f32_u8.cu -- first passes of the sheared forward transform
// (Section 4) over uint8 images: the cyclic pass code with a uint8 source,
// accumulator float.
#include "fht_fused_launch.cuh"

namespace fht {
cudaError_t launch_adjoint_f32_u8(int M, const PassDesc &d, cudaStream_t st) {
    return launch_fused_m<true, float, uint8_t, float, float>(M, d, st);
}
}  // namespace fht
