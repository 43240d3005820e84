// batched_adj_q1.cu -- one instantiation of the persistent batched kernel:
// float adjoints of quadrant Q1: slope sign +, image gradient as is
// (an adjoint runs the opposite sign of its quadrant).
#include "fht_batched.cuh"

namespace fht {
namespace batched {

Kernel kernel_adj_q1(int minb) {
    return minb >= 3 ? batched_kernel<kModeAdj, 1, 3> : batched_kernel<kModeAdj, 1, 2>;
}

}  // namespace batched
}  // namespace fht
