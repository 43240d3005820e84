// fht_kernels.cuh -- device code of one butterfly pass (forward and adjoint).
//
// A work item is one (group, tile) of a pass (see fht_common.cuh): 2^M
// sheared source rows x (tile_w + 2^M - 1) columns are gathered into shared
// memory, M butterfly levels run there, and 2^M rows x tile_w columns are
// written through the destination map. Columns inside a tile are indexed in
// the direction of the shifts ("buffer coordinates"): for sigma = -1 the tile
// is walked right to left, so both signs share one local butterfly:
//   new[2u][i]   = top[u][i] + bot[u][i + u]
//   new[2u+1][i] = top[u][i] + bot[u][i + u + 1].
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

template <typename AccT>
__device__ __forceinline__ AccT load_elem(const void *base, int type, int64_t idx) {
    switch (type) {
    case kU8: return (AccT)((const uint8_t *)base)[idx];
    case kU16: return (AccT)((const uint16_t *)base)[idx];
    case kI32: return (AccT)((const int32_t *)base)[idx];
    default: return (AccT)((const float *)base)[idx];
    }
}

template <typename AccT>
__device__ __forceinline__ void store_elem(void *base, int type, int64_t idx, AccT v,
                                           int accumulate) {
    switch (type) {
    case kU16: ((uint16_t *)base)[idx] = (uint16_t)v; break;
    case kI32: {
        int32_t *p = (int32_t *)base + idx;
        *p = accumulate ? Arith<int32_t>::add(*p, (int32_t)v) : (int32_t)v;
        break;
    }
    default: {
        float *p = (float *)base + idx;
        *p = accumulate ? __fadd_rn(*p, (float)v) : (float)v;
        break;
    }
    }
}

// Level-k0 row of buffer row s in group (S, a); level-k1 row of buffer row c.
__device__ __forceinline__ int lo_row(const PassDesc &d, int M, int S, int a, int s) {
    return d.lo_image ? S * (1 << M) + s : ((S * (1 << M) + s) << d.k0) + a;
}
__device__ __forceinline__ int hi_row(const PassDesc &d, int M, int S, int a, int c) {
    return (S << (d.k0 + M)) + (a << M) + c;
}

// Read the level-k0 value of row `row` at compact column p (zero outside).
template <typename AccT>
__device__ __forceinline__ AccT read_lo(const PassDesc &d, int row, int64_t p) {
    if (d.lo_image) {
        int64_t col = p - (d.sigma > 0 ? 1 : 0);
        if (row >= d.lo.rows || col < 0 || col >= d.lo.cols) return AccT(0);
        int64_t idx = d.transpose ? col * d.lo.pitch + row : (int64_t)row * d.lo.pitch + col;
        return load_elem<AccT>(d.lo.ptr, d.lo.type, idx);
    }
    if (p < 0 || p >= d.lo.cols) return AccT(0);
    return load_elem<AccT>(d.lo.ptr, d.lo.type, (int64_t)row * d.lo.pitch + p);
}

// Output location of a final-level value: returns false if slope t is not
// part of the output. Column X = p - sigma_plus*n (mod W), then fhtshift.
__device__ __forceinline__ bool final_loc(const PassDesc &d, int t, int64_t p,
                                          int64_t *row, int64_t *col) {
    if (t < d.t_first || t > d.t_last) return false;
    int64_t X = p - (d.sigma > 0 ? d.n : 0);
    if (X < 0) X += d.W;
    if (d.shift_on) {
        int s = fhtshift_amount(t, d.W, d.shift_win, d.sigma);
        X = floor_mod(X + (d.shift_inverse ? -s : s), d.W);
    }
    *row = d.row_base + (int64_t)d.row_dir * t;
    *col = X;
    return true;
}

template <typename AccT>
__device__ __forceinline__ AccT read_hi(const PassDesc &d, int row, int64_t p) {
    if (d.hi_final) {
        int64_t r, c;
        if (p < 0 || p >= d.W || !final_loc(d, row, p, &r, &c)) return AccT(0);
        return load_elem<AccT>(d.hi.ptr, d.hi.type, r * d.hi.pitch + c);
    }
    if (p < 0 || p >= d.hi.cols) return AccT(0);
    return load_elem<AccT>(d.hi.ptr, d.hi.type, (int64_t)row * d.hi.pitch + p);
}

template <typename AccT>
__device__ __forceinline__ void write_hi(const PassDesc &d, int row, int64_t p, AccT v) {
    if (d.hi_final) {
        int64_t r, c;
        if (p < 0 || p >= d.W || !final_loc(d, row, p, &r, &c)) return;
        store_elem<AccT>(d.hi.ptr, d.hi.type, r * d.hi.pitch + c, v, 0);
        return;
    }
    if (p < 0 || p >= d.hi.cols) return;
    store_elem<AccT>(d.hi.ptr, d.hi.type, (int64_t)row * d.hi.pitch + p, v, 0);
}

template <typename AccT>
__device__ __forceinline__ void write_lo(const PassDesc &d, int row, int64_t p, AccT v) {
    if (d.lo_image) {
        int64_t col = p - (d.sigma > 0 ? 1 : 0);
        if (row >= d.lo.rows || col < 0 || col >= d.lo.cols) return;
        int64_t idx = d.transpose ? col * d.lo.pitch + row : (int64_t)row * d.lo.pitch + col;
        store_elem<AccT>(d.lo.ptr, d.lo.type, idx, v, d.accumulate);
        return;
    }
    if (p < 0 || p >= d.lo.cols) return;
    store_elem<AccT>(d.lo.ptr, d.lo.type, (int64_t)row * d.lo.pitch + p, v, 0);
}

__host__ __device__ constexpr int round_up4(int v) { return (v + 3) & ~3; }

// Shared memory (elements) of one item: two ping-pong buffers.
__host__ __device__ inline int64_t item_smem_elems(int M, int tile_w) {
    return 2LL * (1 << M) * round_up4(tile_w + (1 << M) - 1);
}

// Forward pass item: levels k0 -> k0 + M of group gy, tile `tile`.
template <int M, typename AccT>
__device__ void forward_item(const PassDesc &d, int gy, int tile, AccT *sm) {
    constexpr int R = 1 << M;
    const int T = d.tile_w;
    const int L = T + R - 1, Lp = round_up4(L);
    AccT *cur = sm, *nxt = sm + R * Lp;
    const int S = gy / d.a_count, a = d.a_lo + gy % d.a_count;
    const int64_t p0 = (int64_t)tile * T;
    const int sg = d.sigma;
    // source column of buffer (s, i): A + sg*(i + a*s); destination column of i: D + sg*i
    const int64_t A = sg > 0 ? p0 - (1LL << (d.k0 + M)) + (1LL << d.k0) : p0 + T - 1;
    const int64_t D = sg > 0 ? p0 : p0 + T - 1;

    for (int idx = threadIdx.x; idx < R * L; idx += blockDim.x) {
        int s = idx / L, i = idx - s * L;
        cur[s * Lp + i] = read_lo<AccT>(d, lo_row(d, M, S, a, s), A + sg * (int64_t)(i + a * s));
    }
    __syncthreads();
#pragma unroll 1
    for (int half = 1; half < R; half *= 2) {
        for (int idx = threadIdx.x; idx < R * L; idx += blockDim.x) {
            int r = idx / L, i = idx - r * L;
            int s0 = r & ~(2 * half - 1), t = r - s0, u = t >> 1;
            int ib = i + u + (t & 1);
            AccT top = cur[(s0 + u) * Lp + i];
            AccT bot = ib < L ? cur[(s0 + half + u) * Lp + ib] : AccT(0);
            nxt[r * Lp + i] = Arith<AccT>::add(top, bot);
        }
        __syncthreads();
        AccT *tmp = cur; cur = nxt; nxt = tmp;
    }
    for (int idx = threadIdx.x; idx < R * T; idx += blockDim.x) {
        int c = idx / T, i = idx - c * T;
        write_hi<AccT>(d, hi_row(d, M, S, a, c), D + sg * (int64_t)i, cur[c * Lp + i]);
    }
    __syncthreads();
}

// Adjoint pass item: the transpose of forward_item (levels k0 + M -> k0).
// Buffer column b holds local column i = b - (R - 1); the split of a merged
// strip sends g[2u] + g[2u+1] to top row u and g[2u](i-u) + g[2u+1](i-u-1)
// to bottom row u.
template <int M, typename AccT>
__device__ void adjoint_item(const PassDesc &d, int gy, int tile, AccT *sm) {
    constexpr int R = 1 << M, H = R - 1;
    const int T = d.tile_w;
    const int L = T + H, Lp = round_up4(L);
    AccT *cur = sm, *nxt = sm + R * Lp;
    const int S = gy / d.a_count, a = d.a_lo + gy % d.a_count;
    const int64_t p0 = (int64_t)tile * T;
    const int sg = d.sigma;
    const int64_t A = sg > 0 ? p0 - (1LL << (d.k0 + M)) + (1LL << d.k0) : p0 + T - 1;
    const int64_t D = sg > 0 ? p0 : p0 + T - 1;

    for (int idx = threadIdx.x; idx < R * L; idx += blockDim.x) {
        int c = idx / L, b = idx - c * L;
        cur[c * Lp + b] = read_hi<AccT>(d, hi_row(d, M, S, a, c), D + sg * (int64_t)(b - H));
    }
    __syncthreads();
#pragma unroll 1
    for (int half = R / 2; half >= 1; half /= 2) {
        for (int idx = threadIdx.x; idx < R * L; idx += blockDim.x) {
            int r = idx / L, b = idx - r * L;
            int s0 = r & ~(2 * half - 1), t = r - s0;
            AccT v;
            if (t < half) {
                v = Arith<AccT>::add(cur[(s0 + 2 * t) * Lp + b], cur[(s0 + 2 * t + 1) * Lp + b]);
            } else {
                int u = t - half;
                AccT g0 = b - u >= 0 ? cur[(s0 + 2 * u) * Lp + b - u] : AccT(0);
                AccT g1 = b - u - 1 >= 0 ? cur[(s0 + 2 * u + 1) * Lp + b - u - 1] : AccT(0);
                v = Arith<AccT>::add(g0, g1);
            }
            nxt[r * Lp + b] = v;
        }
        __syncthreads();
        AccT *tmp = cur; cur = nxt; nxt = tmp;
    }
    for (int idx = threadIdx.x; idx < R * T; idx += blockDim.x) {
        int s = idx / T, i = idx - s * T;
        write_lo<AccT>(d, lo_row(d, M, S, a, s), A + sg * (int64_t)(i + a * s),
                       cur[s * Lp + i + H]);
    }
    __syncthreads();
}

}  // namespace fht
