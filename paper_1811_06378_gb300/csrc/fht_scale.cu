// fht_scale.cu -- the scale of Section 4's angle-range transform: every row
// of the image (of the transposed image for Q2/Q3) resampled by the factor
// alpha with nearest neighbours, written once into the caller's workspace so
// that the first pass of the (sheared) transform reads it with the same
// vector loads as an unscaled image.
//
// The source index of scaled position c is (c * D) >> 32 with the 32.32 step
// D = ceil(2^32 / alpha): for alpha > 1 source pixels repeat, for alpha < 1
// they are skipped. Along the rows of a Q0/Q1 image that is a column gather;
// for Q2/Q3, whose transform reads the image transposed, the scaled axis is
// the image's row index, so every output row is a copy of one source row.
#include <cuda_runtime.h>

#include <cstdint>

#include "fht_common.cuh"
#include "fht_host.h"

namespace fht {
namespace {

constexpr int kScaleThreads = 256;
constexpr int kScalePer = 4;   // consecutive output elements per thread

template <typename T>
struct Pack4;
template <>
struct Pack4<uint8_t> {
    using V = uint32_t;
    __device__ static V make(const uint8_t (&x)[4]) {
        return (uint32_t)x[0] | ((uint32_t)x[1] << 8) | ((uint32_t)x[2] << 16) |
               ((uint32_t)x[3] << 24);
    }
};
template <>
struct Pack4<uint16_t> {
    using V = uint2;
    __device__ static V make(const uint16_t (&x)[4]) {
        return make_uint2((uint32_t)x[0] | ((uint32_t)x[1] << 16),
                          (uint32_t)x[2] | ((uint32_t)x[3] << 16));
    }
};
template <>
struct Pack4<uint32_t> {
    using V = uint4;
    __device__ static V make(const uint32_t (&x)[4]) { return make_uint4(x[0], x[1], x[2], x[3]); }
};

// Output row blockIdx.y, elements c0 .. c0 + 3 of it per thread. The four
// are stored as one vector when the row start and c0 allow it (the
// workspace copy always does), else one by one.
template <typename T, bool ALONG_ROWS>
__global__ void __launch_bounds__(kScaleThreads)
    scale_image_kernel(const T *__restrict__ src, int64_t sp, unsigned long long D,
                       T *__restrict__ dst, int64_t dp, int out_cols) {
    const int r = blockIdx.y;
    const int c0 = (blockIdx.x * kScaleThreads + threadIdx.x) * kScalePer;
    if (c0 >= out_cols) return;
    const T *srow = ALONG_ROWS ? src + (int64_t)(((unsigned long long)r * D) >> 32) * sp
                               : src + (int64_t)r * sp;
    T x[kScalePer];
#pragma unroll
    for (int k = 0; k < kScalePer; ++k) {
        const int c = c0 + k < out_cols ? c0 + k : out_cols - 1;
        const int64_t sc = ALONG_ROWS ? c : (int64_t)(((unsigned long long)c * D) >> 32);
        x[k] = __ldg(srow + sc);
    }
    T *drow = dst + (int64_t)r * dp;
    using V = typename Pack4<T>::V;
    if (c0 + kScalePer <= out_cols &&
        (reinterpret_cast<uintptr_t>(drow + c0) & (sizeof(V) - 1)) == 0) {
        *reinterpret_cast<V *>(drow + c0) = Pack4<T>::make(x);
    } else {
#pragma unroll
        for (int k = 0; k < kScalePer; ++k)
            if (c0 + k < out_cols) drow[c0 + k] = x[k];
    }
}

// uint8 rows, alpha >= 1/2 (D <= 2^33): a block's kSpanOut output columns
// take at most 2 * kSpanOut + 1 consecutive source bytes. The block loads
// that span once into shared memory as aligned 4-byte words (coalesced; the
// source and its pitch are 4-byte aligned, so the words stay inside the
// row's pitch), then every thread gathers 16 output bytes from shared memory
// and stores them as one 16-byte vector.
constexpr int kSpanPer = 16;                              // output bytes per thread
constexpr int kSpanOut = kScaleThreads * kSpanPer;        // output bytes per block
constexpr int kSpanWords = (2 * kSpanOut + 1 + 6) / 4 + 1;  // aligned words of the span

__global__ void __launch_bounds__(kScaleThreads)
    scale_cols_u8_span_kernel(const uint8_t *__restrict__ src, int64_t sp, unsigned long long D,
                              uint8_t *__restrict__ dst, int64_t dp, int out_cols) {
    __shared__ uint32_t span[kSpanWords];
    const int r = blockIdx.y;
    const int b0 = blockIdx.x * kSpanOut;
    const int b1 = (b0 + kSpanOut < out_cols ? b0 + kSpanOut : out_cols) - 1;   // last column
    const long long s_lo = (long long)(((unsigned long long)b0 * D) >> 32);
    const long long s_hi = (long long)(((unsigned long long)b1 * D) >> 32);
    const long long a0 = s_lo & ~3LL;                  // first aligned word (bytes)
    const int nw = (int)(((s_hi + 4) & ~3LL) - a0) / 4;   // words up to the one holding s_hi
    const uint32_t *srow = reinterpret_cast<const uint32_t *>(src + (int64_t)r * sp + a0);
    for (int i = threadIdx.x; i < nw; i += kScaleThreads) span[i] = __ldg(srow + i);
    __syncthreads();
    const uint8_t *sb = reinterpret_cast<const uint8_t *>(span);
    const int c0 = b0 + threadIdx.x * kSpanPer;
    if (c0 >= out_cols) return;
    unsigned long long acc = (unsigned long long)c0 * D;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t word = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + 4 * j + k;
            const long long sc = (long long)(acc >> 32);
            acc += D;
            const uint32_t b = c < out_cols ? (uint32_t)sb[sc - a0] : 0u;
            word |= b << (8 * k);
        }
        w[j] = word;
    }
    uint8_t *drow = dst + (int64_t)r * dp;
    if (c0 + kSpanPer <= out_cols && (reinterpret_cast<uintptr_t>(drow + c0) & 15) == 0) {
        *reinterpret_cast<uint4 *>(drow + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
        for (int k = 0; k < kSpanPer; ++k)
            if (c0 + k < out_cols) drow[c0 + k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
    }
}

template <typename T>
cudaError_t launch_t(const void *src, int64_t sp, bool along_rows, long long D, void *dst,
                     int64_t dp, int out_rows, int out_cols, cudaStream_t st) {
    if constexpr (sizeof(T) == 1) {
        if (!along_rows && (unsigned long long)D <= (1ULL << 33) && sp % 4 == 0 &&
            (reinterpret_cast<uintptr_t>(src) & 3) == 0) {
            const dim3 grid((unsigned)((out_cols + kSpanOut - 1) / kSpanOut), (unsigned)out_rows);
            scale_cols_u8_span_kernel<<<grid, kScaleThreads, 0, st>>>(
                static_cast<const uint8_t *>(src), sp, (unsigned long long)D,
                static_cast<uint8_t *>(dst), dp, out_cols);
            return cudaGetLastError();
        }
    }
    const int per_block = kScaleThreads * kScalePer;
    const dim3 grid((unsigned)((out_cols + per_block - 1) / per_block), (unsigned)out_rows);
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
    if (along_rows)
        scale_image_kernel<T, true>
            <<<grid, kScaleThreads, 0, st>>>(s, sp, (unsigned long long)D, d, dp, out_cols);
    else
        scale_image_kernel<T, false>
            <<<grid, kScaleThreads, 0, st>>>(s, sp, (unsigned long long)D, d, dp, out_cols);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scale_image(const void *src, int64_t src_pitch, int elem, bool along_rows,
                               long long D, void *dst, int64_t dst_pitch, int out_rows,
                               int out_cols, cudaStream_t st) {
    if (out_rows <= 0 || out_cols <= 0) return cudaSuccess;
    if (out_rows > 65535 || D <= 0) return cudaErrorInvalidValue;
    if (elem != 1 && elem != 2 && elem != 4) return cudaErrorInvalidValue;
    // algorithmic bytes: the source pixels used, read once, and the scaled
    // image written once
    const long long last = along_rows ? out_rows - 1 : out_cols - 1;
    const long long used = (long long)(((unsigned long long)last * (unsigned long long)D) >> 32) + 1;
    const double bytes = (double)elem * ((along_rows ? used * out_cols : used * out_rows) +
                                         (double)out_rows * out_cols);
    LaunchScope scope("scale_image", st, bytes);
    cudaError_t e;
    if (elem == 1)
        e = launch_t<uint8_t>(src, src_pitch, along_rows, D, dst, dst_pitch, out_rows, out_cols,
                              st);
    else if (elem == 2)
        e = launch_t<uint16_t>(src, src_pitch, along_rows, D, dst, dst_pitch, out_rows, out_cols,
                               st);
    else
        e = launch_t<uint32_t>(src, src_pitch, along_rows, D, dst, dst_pitch, out_rows, out_cols,
                               st);
    scope.done();
    return e;
}

}  // namespace fht
