// batched_f32_pos.cu -- one instantiation of the persistent batched-forward
// kernel (float, slope sign +).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_f32_pos() { return batched_kernel<kModeF32, 1>; }

}  // namespace batched
}  // namespace fht
