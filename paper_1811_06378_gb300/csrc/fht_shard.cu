// fht_shard.cu -- the last log2(P) butterfly levels of an image whose rows
// are split over P ranks (one strip of n/P rows each).
//
// After its K - log2(P) local levels, strip p holds the level rows
// (strip p, slope tau) for tau < n/P. By the pass identity of the recursion
// (fht_common.cuh), the final slopes tau*P + c (c < P) are the P-row
// transform of the rows (p, tau), p < P, row p read sheared by sigma*tau*p:
//   R_p[x] = L_p[tau][(x + sigma*tau*p) mod W],
//   A_0 = R;  A_{k+1}[s][t][x] = A_k[2s][t/2][x] + A_k[2s+1][t/2][(x + sigma*ceil(t/2)) mod W],
//   H[tau*P + c] = A_log2(P)[0][c],
// the same additions, in the same order, as the recursion's last levels on
// one GPU. A rank that owns the slopes of a block of tau receives those rows
// of every strip (one all-to-all) and runs this kernel on them.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fht.h"
#include "fht_host.h"
#include "fht_kernels.cuh"

namespace {

constexpr int kMergeBlock = 256;

// One thread per (tau, x): the P inputs on the window x .. x + sigma*(P-1)
// (the largest offset of a P-row pattern is P - 1), then the log2(P) levels
// in registers, shrinking the window as the offsets are consumed; output
// rows tau*P + c at column x.
template <int P, typename T>
__global__ void __launch_bounds__(kMergeBlock)
    merge_strips_kernel(const T *parts, int64_t part_stride, int64_t in_pitch, int W, int tau0,
                        int sigma, T *out, int64_t out_pitch) {
    const int x = blockIdx.x * kMergeBlock + threadIdx.x;
    const int r = blockIdx.y;
    if (x >= W) return;
    const int64_t tau = (int64_t)tau0 + r;
    T a[P][P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const T *row = parts + p * part_stride + (int64_t)r * in_pitch;
        int64_t c = ((int64_t)x + sigma * tau * p) % W;
        if (c < 0) c += W;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            a[p][j] = row[c];
            c += sigma;
            if (c == W) c = 0;
            if (c < 0) c = W - 1;
        }
    }
#pragma unroll
    for (int half = 1; half < P; half *= 2) {
        T nv[P][P];
#pragma unroll
        for (int s0 = 0; s0 < P; s0 += 2 * half) {
#pragma unroll
            for (int u = 0; u < half; ++u) {
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    // columns j + u + 1 past the window feed no output
                    nv[s0 + 2 * u][j] =
                        j + u < P ? fht::Arith<T>::add(a[s0 + u][j], a[s0 + half + u][j + u < P ? j + u : 0])
                                  : T(0);
                    nv[s0 + 2 * u + 1][j] =
                        j + u + 1 < P
                            ? fht::Arith<T>::add(a[s0 + u][j],
                                                 a[s0 + half + u][j + u + 1 < P ? j + u + 1 : 0])
                            : T(0);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < P; ++s)
#pragma unroll
            for (int j = 0; j < P; ++j) a[s][j] = nv[s][j];
    }
#pragma unroll
    for (int c = 0; c < P; ++c) out[((int64_t)r * P + c) * out_pitch + x] = a[c][0];
}

template <typename T>
cudaError_t launch_merge(int P, const void *parts, int64_t part_stride, int64_t in_pitch,
                         int rows, int W, int tau0, int sigma, void *out, int64_t out_pitch,
                         cudaStream_t st) {
    const dim3 grid((W + kMergeBlock - 1) / kMergeBlock, rows);
    const T *src = static_cast<const T *>(parts);
    T *dst = static_cast<T *>(out);
    fht::LaunchScope scope("merge_strips", st,
                           (double)rows * W * P * sizeof(T) * 2.0);
    switch (P) {
    case 1:
        merge_strips_kernel<1, T><<<grid, kMergeBlock, 0, st>>>(src, part_stride, in_pitch, W,
                                                              tau0, sigma, dst, out_pitch);
        break;
    case 2:
        merge_strips_kernel<2, T><<<grid, kMergeBlock, 0, st>>>(src, part_stride, in_pitch, W,
                                                              tau0, sigma, dst, out_pitch);
        break;
    case 4:
        merge_strips_kernel<4, T><<<grid, kMergeBlock, 0, st>>>(src, part_stride, in_pitch, W,
                                                              tau0, sigma, dst, out_pitch);
        break;
    default:
        merge_strips_kernel<8, T><<<grid, kMergeBlock, 0, st>>>(src, part_stride, in_pitch, W,
                                                              tau0, sigma, dst, out_pitch);
        break;
    }
    scope.done();
    return cudaGetLastError();
}

}  // namespace

extern "C" fht_status fht_merge_strips(const void *parts, fht_dtype dtype, int strips, int rows,
                                       int W, int64_t part_stride, int64_t in_pitch, int tau0,
                                       fht_quadrant q, void *out, int64_t out_pitch,
                                       void *stream) {
    if (strips != 1 && strips != 2 && strips != 4 && strips != 8) return FHT_EINVAL;
    if (q < FHT_Q0 || q > FHT_Q3 || rows < 0 || W < 1 || tau0 < 0) return FHT_EINVAL;
    if (dtype != FHT_I32 && dtype != FHT_F32) return FHT_EINVAL;
    if (rows == 0) return FHT_OK;
    if (!parts || !out || in_pitch < W || out_pitch < W) return FHT_EINVAL;
    if (strips > 1 && part_stride < (int64_t)rows * in_pitch) return FHT_EINVAL;
    if (rows > 65535) return FHT_EUNSUPPORTED;   // one grid row per tau
    const int sigma = (q == FHT_Q0 || q == FHT_Q3) ? 1 : -1;
    const cudaError_t e =
        dtype == FHT_F32
            ? launch_merge<float>(strips, parts, part_stride, in_pitch, rows, W, tau0, sigma, out,
                                  out_pitch, (cudaStream_t)stream)
            : launch_merge<int32_t>(strips, parts, part_stride, in_pitch, rows, W, tau0, sigma,
                                    out, out_pitch, (cudaStream_t)stream);
    return e == cudaSuccess ? FHT_OK : FHT_ECUDA;
}
