// batched_u8_pos.cu -- one instantiation of the persistent batched-forward
// kernel (uint8 -> int32, slope sign +).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_u8_pos(int minb) {
    return minb >= 3 ? batched_kernel<kModeU8, 1, 3> : batched_kernel<kModeU8, 1, 2>;
}

}  // namespace batched
}  // namespace fht
