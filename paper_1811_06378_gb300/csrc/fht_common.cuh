// fht_common.cuh -- shared definitions of the GB300 fast Hough transform kernels.
//
// Terminology (Brady's dyadic recursion, cited by the paper in Section 2 and
// drawn in Section 4, Figure 6):
//   level k     the array after k butterfly levels: n/2^k strips of 2^k rows,
//               row s*2^k + tau of the array = slope tau of strip s
//   pass        m consecutive levels k0 -> k1 = k0 + m run by one launch.
//
// Pass identity used by every kernel: for a level-k1 strip S and a level-k0
// slope a, the 2^m level-k1 slopes a*2^m + c (c < 2^m) are the m-level
// transform of the 2^m level-k0 rows (S*2^m + s')*2^k0 + a, s' < 2^m, after
// row s' is sheared by sigma*a*s' columns, because
//   off_{2^k1}(a*2^m + c, s'*2^k0 + y) = a*s' + off_{2^m}(c, s') + off_{2^k0}(a, y)
// for y < 2^k0 (expand the closed form: the top m bits of the row index meet
// halvings of a*2^m + c that contribute a*2^(m-j) plus the c-terms). So each
// pass is a set of independent "groups" (S, a), each a small FHT of 2^m
// sheared rows over the full row width, tiled along the columns with a halo
// of 2^m - 1 columns.
//
// Column coordinates. Level-k arrays are stored "compact": column X of the
// cyclic width W is kept at p = (X + sigma_plus * 2^k) mod W, sigma_plus = 1 for
// sigma = +1 and 0 for sigma = -1, and only p < w_c + 2^k is stored (w_c = the
// image's content width): every other column of a level-k array is zero for
// any image. In these coordinates a pass never reads across the cyclic wrap;
// only the final level (2^K = n) maps back to X with one wrap.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fht {

enum ElemType : int { kU8 = 0, kU16 = 1, kI32 = 2, kF32 = 3 };

// One side of a pass: the level-k0 ("lo") or level-k1 ("hi") array.
struct Side {
    void *ptr;
    int64_t pitch;   // elements
    int type;        // ElemType
    int rows;        // lo image: content rows h_c; otherwise n
    int cols;        // lo image: content cols w_c; compact: w_c + 2^k; final: W
};

struct PassDesc {
    Side lo, hi;
    int lo_image;    // lo is the level-0 image (zero outside rows x cols)
    int transpose;   // lo image is read transposed (quadrants Q2, Q3)
    int hi_final;    // hi is the final level: user layout (rows mapped, X columns)
    int n, W, K, k0, sigma;
    // Adjoint passes (the opposite-sign transform of a gradient): every level
    // spans all W columns, read cyclically; the level-0 source is the
    // gradient, row t at src_row_base + src_row_dir*t for t in
    // [src_t_first, src_t_last] and zero otherwise; the final level goes to the
    // image gradient (rows < dst_h, columns < dst_w, transposed if
    // dst_transpose, added to its contents if accumulate).
    int cyclic;
    int src_t_first, src_t_last, src_row_base, src_row_dir;
    int dst_image, dst_h, dst_w, dst_transpose, accumulate;
    int p_begin, p_count;  // destination columns [p_begin, p_begin + p_count) are tiled
    int a_lo, a_count;   // level-k0 slopes of the groups (range pruning)
    // level-k1 slopes [need_lo, need_hi] that later passes or the output use;
    // an item producing none of them is skipped (range pruning inside groups)
    int need_lo, need_hi;
    int s_count;         // strips at level k1
    int tile_w;          // output columns per tile
    int tiles;           // tiles per group
    int n_a;             // fused kernel: block-A warp-columns per tile
    // uniform batch: `batch` same-size transforms in one launch (blockIdx.z),
    // image b's source and destination `b * lo_bstride` / `b * hi_bstride`
    // bytes past lo.ptr / hi.ptr (0 and 1 for a single transform)
    int batch;
    int64_t lo_bstride, hi_bstride;
    int black_wc;        // content width w_c (black-zone test of the final level)
    // final level only: slope t is row row_base + row_dir*t of the output,
    // present for t in [t_first, t_last]
    int t_first, t_last, row_base, row_dir;
    // final level only: fhtshift rotation fused into the row mapping
    int shift_on, shift_win, shift_inverse;
    // Windowed adjoint level: the final pass of an adjoint reads each row of
    // the level before it only on the win_len columns that reach the cropped
    // image gradient, so that level keeps just those. Row (strip s, slope a)
    // holds the columns x of its window, based at win_base(d, s, a), at
    // j = (x - base) mod W < win_len; its pitch is >= win_len + 8. hi_win:
    // this pass writes such a level; lo_win: it reads one.
    int lo_win, hi_win, win_len, win_c;
    // Sheared forward (Section 4), set on every pass of it; it runs on the
    // cyclic (adjoint) pass code with the quadrant's own sign: the level-0
    // source is the (transposed) image whose row y is rotated right by
    // s(y) = (y*shear_p + 2^31) >> 32 columns modulo W (floor(y*spl + 1/2)
    // with spl in 32-bit fixed point, shear_p = floor(spl*2^32 + 1/2)), zero
    // outside its lo.rows x lo.cols content; the final level goes to the
    // quadrant's rows t in [dst_row_lo, dst_h), stored at row t - dst_row_lo.
    int shear_on, dst_row_lo;
    long long shear_p;
    // Host bookkeeping, not read by the kernels: the pass belongs to a range
    // transform (fht_forward_range, fht_forward_op with a slope range), whose
    // launches are named apart from those of whole quadrants.
    int range_call;
    // Bytes from lo.ptr / hi.ptr the pass may touch (0: unknown); read only by
    // the debug build's bounds checks (fht_debug.cuh).
    long long dbg_lo_bytes, dbg_hi_bytes;
};

__host__ __device__ inline int64_t floor_mod(int64_t v, int64_t m) {
    int64_t r = v % m;
    return r < 0 ? r + m : r;
}

// v mod W for v in (-2W, 2W); other values take the general remainder.
__host__ __device__ inline int wrap_w(int v, int W) {
    if (v < 0) v += W;
    if (v >= W) v -= W;
    if ((unsigned)v >= (unsigned)W) {
        v %= W;
        if (v < 0) v += W;
    }
    return v;
}

// First column of the window of level row (strip s, slope a): the final
// pass's group a reads row s sheared by sigma*a*s from column
// win_c + sigma*a*s on, so the window moves with the shear. It starts 8 to 15
// columns before that column, on a multiple of 8: a lane's 8 columns that
// hold any needed column then start inside the window (no wrap), and
// aligned rows stay aligned.
__host__ __device__ inline int win_base_raw(const PassDesc &d, int s, int a) {
    return wrap_w(d.win_c + d.sigma * a * s - 8, d.W);
}
__host__ __device__ inline int win_base(const PassDesc &d, int s, int a) {
    return win_base_raw(d, s, a) & ~7;
}

// fhtshift rotation of slope row t (Section 5): the w_in + t meaningful
// columns start at floor(b/2), b = W - w_in - t; positive-sign quadrants carry
// their meaningful run across the wrap, hence the extra t.
__host__ __device__ inline int fhtshift_amount(int t, int W, int w_in, int sigma) {
    int b = W - w_in - t;
    return b / 2 + (sigma > 0 ? t : 0);
}

}  // namespace fht
