// fht_lines.cu -- from Hough points back to lines: the image segment one
// Hough point sums (Section 3.2) and the per-row maxima of a Hough image
// (where the strongest line of each slope lies).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fht.h"
#include "fht_common.cuh"
#include "fht_host.h"

namespace {

// off_n(t, y) of the dyadic recursion (closed form): the sum over the K bits
// of y, from the top one down, of ceil(floor(t / 2^(j-1)) / 2).
int pattern_offset(int K, int t, int y) {
    int off = 0;
    for (int j = 1; j <= K; ++j)
        if ((y >> (K - j)) & 1) off += ((t >> (j - 1)) + 1) >> 1;
    return off;
}

int next_pow2_i(int v) {
    int n = 1;
    while (n < v) n *= 2;
    return n;
}

constexpr int kArgBlock = 256;

// One block per row: the row's maximum and the first column holding it.
// Each thread scans a strided part of the row, then a shared-memory
// reduction keeps (value, column) with ties going to the smaller column.
template <typename T>
__global__ void __launch_bounds__(kArgBlock)
    row_argmax_kernel(const T *in, int cols, int64_t pitch, T *max_out, int *arg_out) {
    __shared__ T s_v[kArgBlock];
    __shared__ int s_i[kArgBlock];
    const T *row = in + (int64_t)blockIdx.x * pitch;
    T best = row[0];
    int bi = 0;
    for (int c = threadIdx.x; c < cols; c += kArgBlock) {
        const T v = row[c];
        if (v > best || (v == best && c < bi)) {
            best = v;
            bi = c;
        }
    }
    s_v[threadIdx.x] = best;
    s_i[threadIdx.x] = bi;
    __syncthreads();
    for (int half = kArgBlock / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half) {
            const T v = s_v[threadIdx.x + half];
            const int i = s_i[threadIdx.x + half];
            if (v > s_v[threadIdx.x] || (v == s_v[threadIdx.x] && i < s_i[threadIdx.x])) {
                s_v[threadIdx.x] = v;
                s_i[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        max_out[blockIdx.x] = s_v[0];
        arg_out[blockIdx.x] = s_i[0];
    }
}

}  // namespace

extern "C" {

fht_status fht_segment(int h, int w, fht_layout layout, fht_quadrant q, int row, int col,
                       int shifted, int *count, int *r0, int *c0, int *r1, int *c1) {
    if (h < 1 || w < 1 || h > 32768 || w > 32768 || !count || !r0 || !c0 || !r1 || !c1)
        return FHT_EINVAL;
    int qq = q, t = row, n, W, hq, wq;   // quadrant, slope, geometry of its (padded) image
    if (layout == FHT_LAYOUT_FULL) {
        int fq = 0;
        if (fht_full_row_to_quadrant(h, w, row, &fq, &t) != FHT_OK) return FHT_EINVAL;
        qq = fq;
        const int hp = next_pow2_i(h), wp = next_pow2_i(w);
        hq = qq >= 2 ? wp : hp;   // rows of the (transposed) padded image
        wq = qq >= 2 ? hp : wp;
        n = hq;
        W = hp + wp;
    } else if (layout == FHT_LAYOUT_QUADRANT) {
        if (q < 0 || q > 3) return FHT_EINVAL;
        hq = q >= 2 ? w : h;
        wq = q >= 2 ? h : w;
        n = next_pow2_i(hq);
        W = wq + n;
        if (t < 0 || t >= n) return FHT_EINVAL;
    } else {
        return FHT_EINVAL;
    }
    if (col < 0 || col >= W) return FHT_EINVAL;
    const int sigma = (qq == 0 || qq == 3) ? 1 : -1;
    const bool tr = qq >= 2;
    int x = col;
    if (shifted) {
        // undo fhtshift (Section 5): the point came from column x - s(t)
        const int w_in = layout == FHT_LAYOUT_FULL ? W - n : wq;
        x = (int)fht::floor_mod((int64_t)x - fht::fhtshift_amount(t, W, w_in, sigma), W);
    }
    // the image itself (h x w), seen as the (transposed) quadrant's rows and columns
    const int rows_in = tr ? w : h, cols_in = tr ? h : w;
    int K = 0;
    while ((1 << K) < n) ++K;
    int cnt = 0, ya = -1, ca = -1, yb = -1, cb = -1;
    for (int y = 0; y < rows_in && y < n; ++y) {
        const int c = (int)fht::floor_mod((int64_t)x + sigma * pattern_offset(K, t, y), W);
        if (c < cols_in) {
            if (cnt == 0) { ya = y; ca = c; }
            yb = y;
            cb = c;
            ++cnt;
        }
    }
    *count = cnt;
    if (cnt == 0) {
        *r0 = *c0 = *r1 = *c1 = -1;
        return FHT_OK;
    }
    if (tr) {
        *r0 = ca; *c0 = ya; *r1 = cb; *c1 = yb;
    } else {
        *r0 = ya; *c0 = ca; *r1 = yb; *c1 = cb;
    }
    return FHT_OK;
}

fht_status fht_row_argmax(const void *hough, fht_dtype dtype, int rows, int cols, int64_t pitch,
                          void *max_out, int *arg_out, void *stream) {
    if (!hough || !max_out || !arg_out || rows < 0 || cols < 1 || pitch < cols)
        return FHT_EINVAL;
    if (dtype != FHT_I32 && dtype != FHT_F32) return FHT_EINVAL;
    if (rows == 0) return FHT_OK;
    if (rows > 0x7fffffff / 2) return FHT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    fht::LaunchScope scope(dtype == FHT_I32 ? "row_argmax_i32" : "row_argmax_f32", st,
                           (double)rows * cols * 4.0);
    if (dtype == FHT_I32)
        row_argmax_kernel<int32_t><<<rows, kArgBlock, 0, st>>>(
            static_cast<const int32_t *>(hough), cols, pitch, static_cast<int32_t *>(max_out),
            arg_out);
    else
        row_argmax_kernel<float><<<rows, kArgBlock, 0, st>>>(
            static_cast<const float *>(hough), cols, pitch, static_cast<float *>(max_out),
            arg_out);
    scope.done();
    return cudaGetLastError() == cudaSuccess ? FHT_OK : FHT_ECUDA;
}

}  // extern "C"
