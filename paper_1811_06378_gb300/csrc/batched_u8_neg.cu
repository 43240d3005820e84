// batched_u8_neg.cu -- one instantiation of the persistent batched-forward
// kernel (uint8 -> int32, slope sign -).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_u8_neg() { return batched_kernel<kModeU8, -1>; }

}  // namespace batched
}  // namespace fht
