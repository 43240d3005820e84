// batched_f32_neg.cu -- one instantiation of the persistent batched-forward
// kernel (float, slope sign -).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_f32_neg(int minb) {
    return minb >= 3 ? batched_kernel<kModeF32, -1, 3> : batched_kernel<kModeF32, -1, 2>;
}

}  // namespace batched
}  // namespace fht
