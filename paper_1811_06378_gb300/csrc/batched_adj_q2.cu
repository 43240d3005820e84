// batched_adj_q2.cu -- one instantiation of the persistent batched kernel:
// float adjoints of quadrant Q2: slope sign +, image gradient transposed
// (an adjoint runs the opposite sign of its quadrant).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_adj_q2(int minb) {
    return minb >= 3 ? batched_kernel<kModeAdjT, 1, 3> : batched_kernel<kModeAdjT, 1, 2>;
}

}  // namespace batched
}  // namespace fht
