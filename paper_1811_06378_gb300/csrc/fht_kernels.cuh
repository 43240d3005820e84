// fht_kernels.cuh -- arithmetic and row-index helpers shared by the pass kernels.
#pragma once

#include "fht_common.cuh"

namespace fht {

template <typename T> struct Arith;
template <> struct Arith<int32_t> {
    // integer accumulation wraps modulo 2^32
    __device__ static int32_t add(int32_t a, int32_t b) {
        return (int32_t)((uint32_t)a + (uint32_t)b);
    }
};
template <> struct Arith<float> {
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
};

// The operation along the patterns: OP 0 the sum (Arith), 1 the maximum, 2 the
// minimum (the recursion's operands in order: top, then the shifted bottom).
template <typename T, int OP> struct Combine {
    __device__ static T apply(T a, T b) { return Arith<T>::add(a, b); }
};
template <typename T> struct Combine<T, 1> {
    __device__ static T apply(T a, T b) { return a > b ? a : b; }
};
template <typename T> struct Combine<T, 2> {
    __device__ static T apply(T a, T b) { return a < b ? a : b; }
};

// Level-k1 row of output row c of group (S, a) in a pass of M levels.
__device__ __forceinline__ int hi_row(const PassDesc &d, int M, int S, int a, int c) {
    return (S << (d.k0 + M)) + (a << M) + c;
}

}  // namespace fht
