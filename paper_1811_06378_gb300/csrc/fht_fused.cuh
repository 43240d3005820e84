// fht_fused.cuh -- register-level butterfly pass (forward) for sm_103a.
//
// One CTA computes one (group, tile) of a pass of m = MA + MB levels
// (see fht_common.cuh for groups, the pass identity and compact columns).
// Inside the tile, columns run in the direction of the shifts ("buffer
// coordinates"), so both signs use one butterfly.
//
// Data placement:
//  * a lane owns kV = 8 consecutive buffer columns of 2^MA (or 2^MB) rows in
//    registers; a level's shift reaches at most 4 columns into lane+1's
//    registers, fetched with warp shuffles. A warp therefore produces valid
//    results for lanes 0..30 (248 columns); warps overlap by one lane.
//  * block A (levels 0..MA): rows g*2^MA + rho of the group's 2^m sheared
//    source rows, loaded straight from global memory with 8/16-byte vectors
//    and realigned in registers without branches; results go to a shared tile.
//  * block B (levels MA..m): rows g*2^MA + a' (g < 2^MB) read from the tile
//    with the local shear a'*g (the pass identity applied inside the pass),
//    stored to global memory through the destination map.
//  * the shared tile is padded by one 4-byte word (or two 2-byte elements) per
//    8 columns: lanes 8 columns apart then sit 9 words (5 words) apart, so
//    block A's stores and block B's sheared loads are bank-conflict-free and
//    use immediate offsets from one base address per row.
#pragma once

#include <type_traits>

#include "fht_debug.cuh"
#include "fht_kernels.cuh"

namespace fht {

constexpr int kV = 8;                         // columns per lane
constexpr int kLanesValid = 31;               // lanes whose results are complete
constexpr int kWarpValid = kV * kLanesValid;  // 248 columns per warp

template <typename T>
__device__ __forceinline__ T shfl_next(T v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// ------------------------------------------------------------ shared tile

template <typename MidE>
struct TilePad {
    static constexpr int kPad = sizeof(MidE) == 2 ? 2 : 1;   // elements per 8 columns
};

__host__ __device__ inline int tile_pos(int x, int pad) { return x + pad * (x >> 3); }

// ------------------------------------------------------------ global row segments

__device__ __forceinline__ uint32_t sel4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, int j) {
    uint32_t lo = (j & 1) ? b : a;
    uint32_t hi = (j & 1) ? d : c;
    return (j & 2) ? hi : lo;
}

template <typename Acc>
__device__ __forceinline__ Acc from_word(uint32_t w, std::true_type /*float*/) {
    return __uint_as_float(w);
}
template <typename Acc>
__device__ __forceinline__ Acc from_word(uint32_t w, std::false_type) {
    return (Acc)(int32_t)w;
}

// Low halves of lo and hi as one word (lo in bits 0..15): one byte permute.
__device__ __forceinline__ uint32_t pack_u16x2(uint32_t lo, uint32_t hi) {
    return __byte_perm(lo, hi, 0x5410u);
}

// Eight values passed by value to and from the out-of-line edge paths.
template <typename Acc>
struct Vec8 {
    Acc x[8];
};

// Edge paths (tile borders, wraps, unaligned rows) are rare; keeping them out
// of line keeps the hot loop small enough for the instruction cache.
template <typename E, typename Acc>
__device__ __noinline__ Vec8<Acc> load8_edge(const E *row, int lo, int cols) {
    Vec8<Acc> r;
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int c = lo + k;
        r.x[k] = (c >= 0 && c < cols && FHT_LOAD_OK(row + c, sizeof(E))) ? (Acc)row[c] : Acc(0);
    }
    return r;
}

template <typename E, typename Acc>
__device__ __noinline__ void store8_edge(E *row, int lo, int cols, Vec8<Acc> v) {
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int c = lo + k;
        if (c >= 0 && c < cols && FHT_STORE_OK(row + c, sizeof(E))) row[c] = (E)v.x[k];
    }
}

// One aligned vector load. NC (the default) reads through the non-coherent
// read-only path (ld.global.nc), which CUDA allows only for data that no
// thread writes during the kernel: the caller's images and gradients, and
// levels written by an earlier launch. A level written earlier in the same
// launch (the persistent batched kernel, whose passes hand levels to each
// other through its dependency counters) must be read with NC = false: a
// plain, coherent load, ordered after the producer's release by the
// consumer's acquire.
template <bool NC, typename V>
__device__ __forceinline__ V ldvec(const V *p) {
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// v[k] = row[lo + k] for k < 8; all 8 must lie inside the row. The aligned
// granules covering them are loaded whole; the start offset inside the first
// granule selects the elements with selects and byte permutes (no branches,
// so the loads of several rows can all be in flight together).
template <typename E, typename Acc, bool NC = true>
__device__ __forceinline__ void load8_fast(const E *row, int lo, Acc (&v)[kV]) {
    if (!FHT_LOAD_OK(row + lo, kV * sizeof(E))) {
#pragma unroll
        for (int k = 0; k < kV; ++k) v[k] = Acc(0);
        return;
    }
    const uintptr_t a = reinterpret_cast<uintptr_t>(row + lo);
    if constexpr (sizeof(E) == 1) {
        const int delta = (int)(a & 7);
        const uint2 *g = reinterpret_cast<const uint2 *>(a & ~(uintptr_t)7);
        uint2 q0 = ldvec<NC>(g), q1 = make_uint2(0, 0);
        if (delta) q1 = ldvec<NC>(g + 1);
        const uint32_t w0 = q0.x, w1 = q0.y, w2 = q1.x, w3 = q1.y;
        const bool hi = delta >= 4;
        const uint32_t u0 = hi ? w1 : w0, u1 = hi ? w2 : w1, u2 = hi ? w3 : w2;
        const uint32_t sel = 0x3210u + 0x1111u * (uint32_t)(delta & 3);
        const uint32_t b0 = __byte_perm(u0, u1, sel), b1 = __byte_perm(u1, u2, sel);
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // byte k, zero-extended: one byte permute each
            v[k] = (Acc)(int32_t)__byte_perm(b0, 0u, 0x4440u | k);
            v[k + 4] = (Acc)(int32_t)__byte_perm(b1, 0u, 0x4440u | k);
        }
    } else if constexpr (sizeof(E) == 2) {
        const int delta = (int)((a & 15) >> 1);
        const uint4 *g = reinterpret_cast<const uint4 *>(a & ~(uintptr_t)15);
        uint4 q0 = ldvec<NC>(g), q1 = make_uint4(0, 0, 0, 0);
        if (delta) q1 = ldvec<NC>(g + 1);
        const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        const int j = delta >> 1;
        uint32_t u[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) u[i] = sel4(w[i], w[i + 1 < 8 ? i + 1 : 7],
                                              w[i + 2 < 8 ? i + 2 : 7], w[i + 3 < 8 ? i + 3 : 7], j);
        const uint32_t sel = (delta & 1) ? 0x5432u : 0x3210u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t pr = __byte_perm(u[i], u[i + 1], sel);
            v[2 * i] = (Acc)(int32_t)(pr & 0xffffu);
            v[2 * i + 1] = (Acc)(int32_t)(pr >> 16);
        }
    } else {
        const int delta = (int)((a & 15) >> 2);
        const uint4 *g = reinterpret_cast<const uint4 *>(a & ~(uintptr_t)15);
        uint4 q0 = ldvec<NC>(g), q1 = ldvec<NC>(g + 1), q2 = make_uint4(0, 0, 0, 0);
        if (delta) q2 = ldvec<NC>(g + 2);
        const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y,
                                q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
        using IsF = std::integral_constant<bool, std::is_same<Acc, float>::value &&
                                                     std::is_same<E, float>::value>;
#pragma unroll
        for (int k = 0; k < kV; ++k)
            v[k] = from_word<Acc>(sel4(w[k], w[k + 1], w[k + 2], w[k + 3], delta), IsF());
    }
}

// v[k] = p[k] for k < 8, p on a vector granule (8 bytes for uint8, 16
// otherwise) and all 8 in bounds: whole vectors, no realignment.
template <typename E, typename Acc, bool NC = true>
__device__ __forceinline__ void load8_aligned(const E *p, Acc (&v)[kV]) {
    if (!FHT_LOAD_OK(p, kV * sizeof(E))) {
#pragma unroll
        for (int k = 0; k < kV; ++k) v[k] = Acc(0);
        return;
    }
    if constexpr (sizeof(E) == 1) {
        const uint2 q = ldvec<NC>(reinterpret_cast<const uint2 *>(p));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (Acc)(int32_t)__byte_perm(q.x, 0u, 0x4440u | k);
            v[k + 4] = (Acc)(int32_t)__byte_perm(q.y, 0u, 0x4440u | k);
        }
    } else if constexpr (sizeof(E) == 2) {
        const uint4 q = ldvec<NC>(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = (Acc)(int32_t)(w[i] & 0xffffu);
            v[2 * i + 1] = (Acc)(int32_t)(w[i] >> 16);
        }
    } else {
        const uint4 q0 = ldvec<NC>(reinterpret_cast<const uint4 *>(p));
        const uint4 q1 = ldvec<NC>(reinterpret_cast<const uint4 *>(p) + 1);
        const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        using IsF = std::integral_constant<bool, std::is_same<Acc, float>::value &&
                                                     std::is_same<E, float>::value>;
#pragma unroll
        for (int k = 0; k < kV; ++k) v[k] = from_word<Acc>(w[k], IsF());
    }
}

// v[k] = row[lo + k] for k < 8, zero outside [0, cols).
template <typename E, typename Acc, bool NC = true>
__device__ __forceinline__ void load8(const E *row, int lo, int cols, Acc (&v)[kV]) {
    if (lo >= 0 && lo + kV <= cols) {
        load8_fast<E, Acc, NC>(row, lo, v);
    } else {
        const Vec8<Acc> r = load8_edge<E, Acc>(row, lo, cols);
#pragma unroll
        for (int k = 0; k < kV; ++k) v[k] = r.x[k];
    }
}

// Cyclic variant: v[k] = row[(lo + k) mod W] (gradients have no zero zone).
template <typename E, typename Acc, bool NC = true>
__device__ __forceinline__ void load8_cyclic(const E *row, int lo, int W, Acc (&v)[kV]) {
    int c = lo;
    if (c < 0 || c >= W) {
        c %= W;
        if (c < 0) c += W;
    }
    if (c + kV <= W) {
        load8<E, Acc, NC>(row, c, W, v);
        return;
    }
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        int x = c + k;
        if (x >= W) x -= W;
        if (x >= W) x %= W;
        v[k] = FHT_LOAD_OK(row + x, sizeof(E)) ? (Acc)row[x] : Acc(0);
    }
}

template <typename Acc>
__device__ __forceinline__ void reverse8(Acc (&v)[kV]) {
#pragma unroll
    for (int k = 0; k < kV / 2; ++k) {
        Acc t = v[k];
        v[k] = v[kV - 1 - k];
        v[kV - 1 - k] = t;
    }
}

// Store 8 ascending elements at row[lo..lo+7], dropping those outside [0, cols).
// kStream marks data no later pass of this transform reads (the final level):
// its vector stores are evict-first in L2, so they displace less of the
// intermediate level the pass is reading.
template <typename E, typename Acc, bool kStream = false>
__device__ __forceinline__ void store8(E *row, int lo, int cols, const Acc (&v)[kV]) {
    E *p = row + lo;
    if (lo >= 0 && lo + kV <= cols && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        if (!FHT_STORE_OK(p, kV * sizeof(E))) return;
        if constexpr (sizeof(E) == 2) {
            uint4 q;
            q.x = pack_u16x2((uint32_t)v[0], (uint32_t)v[1]);
            q.y = pack_u16x2((uint32_t)v[2], (uint32_t)v[3]);
            q.z = pack_u16x2((uint32_t)v[4], (uint32_t)v[5]);
            q.w = pack_u16x2((uint32_t)v[6], (uint32_t)v[7]);
            if constexpr (kStream) __stcs(reinterpret_cast<uint4 *>(p), q);
            else *reinterpret_cast<uint4 *>(p) = q;
        } else {
            using V4 = typename std::conditional<std::is_same<E, float>::value, float4, int4>::type;
            V4 a, b;
            a.x = (E)v[0]; a.y = (E)v[1]; a.z = (E)v[2]; a.w = (E)v[3];
            b.x = (E)v[4]; b.y = (E)v[5]; b.z = (E)v[6]; b.w = (E)v[7];
            if constexpr (kStream) {
                __stcs(reinterpret_cast<V4 *>(p), a);
                __stcs(reinterpret_cast<V4 *>(p) + 1, b);
            } else {
                reinterpret_cast<V4 *>(p)[0] = a;
                reinterpret_cast<V4 *>(p)[1] = b;
            }
        }
    } else {
        Vec8<Acc> r;
#pragma unroll
        for (int k = 0; k < kV; ++k) r.x[k] = v[k];
        store8_edge<E, Acc>(row, lo, cols, r);
    }
}

// 8 ascending elements to p[0..7], p 16-byte aligned and the 8 columns in
// bounds (the caller checked both once for all its rows).
template <typename E, typename Acc, bool kStream = false>
__device__ __forceinline__ void store8_vec(E *p, const Acc (&v)[kV]) {
    if (!FHT_STORE_OK(p, kV * sizeof(E))) return;
    if constexpr (sizeof(E) == 2) {
        uint4 q;
        q.x = pack_u16x2((uint32_t)v[0], (uint32_t)v[1]);
        q.y = pack_u16x2((uint32_t)v[2], (uint32_t)v[3]);
        q.z = pack_u16x2((uint32_t)v[4], (uint32_t)v[5]);
        q.w = pack_u16x2((uint32_t)v[6], (uint32_t)v[7]);
        if constexpr (kStream) __stcs(reinterpret_cast<uint4 *>(p), q);
        else *reinterpret_cast<uint4 *>(p) = q;
    } else {
        using V4 = typename std::conditional<std::is_same<E, float>::value, float4, int4>::type;
        V4 a, b;
        a.x = (E)v[0]; a.y = (E)v[1]; a.z = (E)v[2]; a.w = (E)v[3];
        b.x = (E)v[4]; b.y = (E)v[5]; b.z = (E)v[6]; b.w = (E)v[7];
        if constexpr (kStream) {
            __stcs(reinterpret_cast<V4 *>(p), a);
            __stcs(reinterpret_cast<V4 *>(p) + 1, b);
        } else {
            reinterpret_cast<V4 *>(p)[0] = a;
            reinterpret_cast<V4 *>(p)[1] = b;
        }
    }
}

// ------------------------------------------------------------ register butterfly

// MR levels on 2^MR rows x 8 columns held by this lane; a bottom row's shifted
// columns past this lane's 8 come from lane+1 (lane 31 receives lane 0's,
// which only ever reaches lane 31's own discarded results).
template <int MR, typename Acc, int OP = 0>
__device__ __forceinline__ void reg_butterfly(Acc (&v)[1 << MR][kV]) {
    constexpr int R = 1 << MR;
#pragma unroll
    for (int half = 1; half < R; half *= 2) {
        Acc nv[R][kV];
#pragma unroll
        for (int s0 = 0; s0 < R; s0 += 2 * half) {
#pragma unroll
            for (int u = 0; u < half; ++u) {
                const Acc *top = v[s0 + u];
                const Acc *bot = v[s0 + half + u];
                Acc nb[kV];
#pragma unroll
                for (int k = 0; k < kV; ++k) nb[k] = k <= u ? shfl_next(bot[k]) : Acc(0);
#pragma unroll
                for (int k = 0; k < kV; ++k) {
                    Acc b0 = k + u < kV ? bot[k + u] : nb[k + u - kV];
                    Acc b1 = k + u + 1 < kV ? bot[k + u + 1] : nb[k + u + 1 - kV];
                    nv[s0 + 2 * u][k] = Combine<Acc, OP>::apply(top[k], b0);
                    nv[s0 + 2 * u + 1][k] = Combine<Acc, OP>::apply(top[k], b1);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < kV; ++k) v[r][k] = nv[r][k];
    }
}

}  // namespace fht

#include "fht_packed.cuh"

namespace fht {

// ------------------------------------------------------------ pass geometry

// Tile geometry of a pass with levels MA + MB (host and device agree on it).
struct TileGeom {
    int tile_out;    // output columns per tile
    int n_a, n_b;    // warp-columns of blocks A and B
    int cols;        // tile columns block B may read
    int pitch;       // shared-memory row pitch (elements, padded), 0 if no tile
};

__host__ __device__ inline TileGeom tile_geom(int MA, int MB, int n_a, int nwarps, int pad) {
    TileGeom g{};
    if (MB == 0) {
        g.n_a = nwarps;
        g.tile_out = nwarps * kWarpValid;
        return g;
    }
    const int RA = 1 << MA, RB = 1 << MB;
    // block B's last valid lane reaches (RB-1) + (RA-1)(RB-1) columns past the
    // tile: those must lie inside block A's valid columns
    const int reach = (RB - 1) * RA;
    g.n_a = n_a;
    g.tile_out = (n_a * kWarpValid - reach) / kV * kV;
    g.n_b = (g.tile_out + kWarpValid - 1) / kWarpValid;
    // highest column block B loads (+1): lanes past the tile read as the
    // first lane past it (tile_block_b), which is the last one a stored
    // lane takes shuffled columns from; one granule more for the pad
    const int max_col = g.tile_out + (RA - 1) * (RB - 1) + kV + 1;
    g.cols = (max_col > n_a * kWarpValid ? max_col : n_a * kWarpValid);
    g.cols = (g.cols + 7) & ~7;
    g.pitch = (tile_pos(g.cols, pad) + 7) & ~7;
    return g;
}

// ------------------------------------------------------------ the pass item

// Source row segment for block A: 8 buffer columns starting at i0 of buffer
// row s, into v (buffer order).
template <int SG, bool ADJ, typename Acc, typename SrcE, bool NC = true>
__device__ __forceinline__ void load_source(const PassDesc &d, int M, int S, int a, int s,
                                            int A_off, int i0, Acc (&v)[kV]) {
    constexpr int sg = SG;
    const int p_first = A_off + sg * (i0 + a * s);
    const int lo = sg > 0 ? p_first : p_first - (kV - 1);
    const SrcE *base = reinterpret_cast<const SrcE *>(d.lo.ptr);
    if (d.lo_image) {
        int row = S * (1 << M) + s;
        const int col = lo - (sg > 0 ? 1 : 0);
        if constexpr (ADJ) {
            // gradient rows through the layout's row map
            if (row < d.src_t_first || row > d.src_t_last) {
#pragma unroll
                for (int k = 0; k < kV; ++k) v[k] = Acc(0);
                return;
            }
            row = d.src_row_base + d.src_row_dir * row;
            load8_cyclic<SrcE, Acc, NC>(base + (int64_t)row * d.lo.pitch, col, d.W, v);
        } else {
            if (row >= d.lo.rows) {
#pragma unroll
                for (int k = 0; k < kV; ++k) v[k] = Acc(0);
                return;
            }
            load8<SrcE, Acc, NC>(base + (int64_t)row * d.lo.pitch, col, d.lo.cols, v);
        }
    } else {
        const int row = ((S * (1 << M) + s) << d.k0) + a;
        if constexpr (ADJ) load8_cyclic<SrcE, Acc, NC>(base + (int64_t)row * d.lo.pitch, lo, d.W, v);
        else load8<SrcE, Acc, NC>(base + (int64_t)row * d.lo.pitch, lo, d.lo.cols, v);
    }
    if (sg < 0) reverse8(v);
}

// Transposed image block for block A of the first pass (quadrants Q2, Q3):
// rows s0..s0+RA-1 of the transposed image are image columns; the 8 buffer
// columns are 8 image rows.
template <int SG, int RA, typename Acc, typename SrcE, bool NC = true>
__device__ __forceinline__ void load_source_transposed(const PassDesc &d, int M, int S,
                                                       int s0, int A_off, int i0,
                                                       Acc (&v)[RA][kV]) {
    constexpr int sg = SG;
    const int p_first = A_off + sg * i0;
    const int lo = (sg > 0 ? p_first : p_first - (kV - 1)) - (sg > 0 ? 1 : 0);  // image row
    const int y0 = S * (1 << M) + s0;                                         // image column
    const SrcE *img = reinterpret_cast<const SrcE *>(d.lo.ptr);
    Acc blk[kV][kV];   // blk[k][j]: image row lo + k, image column y0 + j
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int c = lo + k;   // image row
        if (c >= 0 && c < d.lo.cols) {
            load8<SrcE, Acc, NC>(img + (int64_t)c * d.lo.pitch, y0, d.lo.rows, blk[k]);
        } else {
#pragma unroll
            for (int j = 0; j < kV; ++j) blk[k][j] = Acc(0);
        }
    }
    // buffer order: ascending image rows for sigma = +1, descending otherwise
#pragma unroll
    for (int r = 0; r < RA; ++r)
#pragma unroll
        for (int k = 0; k < kV; ++k) v[r][k] = sg > 0 ? blk[k][r] : blk[kV - 1 - k][r];
}

// ------------------------------------------------------------ block A source

template <typename Acc, int R>
struct Block {
    Acc x[R][kV];
};

// Rare edge items (tile borders, image borders, wraps): per-row checked loads,
// out of line.
template <int SG, int RA, bool ADJ, typename Acc, typename SrcE, bool NC = true>
__device__ __noinline__ Block<Acc, RA> load_block_a_edge(const PassDesc &d, int M, int S, int a,
                                                         int s0, int A_off, int i0) {
    Block<Acc, RA> b;
    if (!ADJ && d.lo_image && d.transpose) {
        load_source_transposed<SG, RA, Acc, SrcE, NC>(d, M, S, s0, A_off, i0, b.x);
    } else {
#pragma unroll
        for (int r = 0; r < RA; ++r)
            load_source<SG, ADJ, Acc, SrcE, NC>(d, M, S, a, s0 + r, A_off, i0, b.x[r]);
    }
    return b;
}

// Shift of sheared image row y: floor(y*spl + 1/2) on the 32-bit fixed-point
// spl, exact in 64-bit integers (|y * shear_p| < 2^47).
__device__ __forceinline__ int shear_shift(const PassDesc &d, int y) {
    return (int)(((long long)y * d.shear_p + (1LL << 31)) >> 32);
}

// Rare sheared loads: the 8 columns wrap past W, or the image is read
// transposed (8 image rows of one column).
template <typename Acc, typename SrcE>
__device__ __noinline__ Vec8<Acc> load8_sheared_edge(const PassDesc &d, const SrcE *img, int y,
                                                     int c0) {
    Vec8<Acc> r;
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        int c = c0 + k;
        if (c >= d.W) c -= d.W;
        Acc v = Acc(0);
        const SrcE *q = d.transpose ? img + (int64_t)c * d.lo.pitch + y
                                    : img + (int64_t)y * d.lo.pitch + c;
        if (c < d.lo.cols && FHT_LOAD_OK(q, sizeof(SrcE))) v = (Acc)*q;
        r.x[k] = v;
    }
    return r;
}

// Block A's source rows of a sheared forward's first pass: image row
// row0 + r (an image column for the transposed quadrants) rotated right by
// its shear shift, cyclically on W, zero outside the image; this lane's 8
// ascending columns start at X (buffer order after the reverse for sign -1).
template <int SG, int RA, typename Acc, typename SrcE, bool NC = true>
__device__ __forceinline__ void load_block_a_sheared(const PassDesc &d, int row0, int X,
                                                     int Xw0, int Xw1, Acc (&v)[RA][kV]) {
    const SrcE *img = reinterpret_cast<const SrcE *>(d.lo.ptr);
    if (!d.transpose && row0 + RA <= d.lo.rows) {
        // Whether every row's columns for the whole warp ([Xw0, Xw1) less the
        // row's shift) lie inside the image is decided once, warp-uniformly,
        // from the first and last row (the shifts are monotone in y); then all
        // rows' loads are issued without branches.
        const int sa = shear_shift(d, row0), sb = shear_shift(d, row0 + RA - 1);
        const int s_lo = sa < sb ? sa : sb, s_hi = sa < sb ? sb : sa;
        if (Xw0 - s_hi >= 0 && Xw1 - s_lo <= d.lo.cols) {
            const SrcE *p0 = img + (int64_t)row0 * d.lo.pitch;
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                load8_fast<SrcE, Acc, NC>(p0 + r * d.lo.pitch, X - shear_shift(d, row0 + r), v[r]);
                if constexpr (SG < 0) reverse8(v[r]);
            }
            return;
        }
    }
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        const int y = row0 + r;
        if (y >= d.lo.rows) {
#pragma unroll
            for (int k = 0; k < kV; ++k) v[r][k] = Acc(0);
            continue;
        }
        const int c0 = wrap_w(X - shear_shift(d, y), d.W);
        if (!d.transpose && c0 + kV <= d.W) {
            load8<SrcE, Acc, NC>(img + (int64_t)y * d.lo.pitch, c0, d.lo.cols, v[r]);
        } else {
            const Vec8<Acc> e = load8_sheared_edge<Acc, SrcE>(d, img, y, c0);
#pragma unroll
            for (int k = 0; k < kV; ++k) v[r][k] = e.x[k];
        }
        if constexpr (SG < 0) reverse8(v[r]);
    }
}

// Block A's RA source rows s0.. for this lane's 8 buffer columns i0..i0+7.
// Whether every row and every lane of the warp item (columns wbase ..
// wbase + 255) lies inside the source is decided once, warp-uniformly; the
// common interior case then issues all rows' loads without branches.
template <int SG, int RA, bool ADJ, typename Acc, typename SrcE, bool NC = true>
__device__ __forceinline__ void load_block_a(const PassDesc &d, int M, int S, int a, int s0,
                                             int A_off, int wbase, int i0, Acc (&v)[RA][kV]) {
    constexpr int sg = SG;
    const int splus = sg > 0 ? 1 : 0;
    if constexpr (ADJ) {
        if (d.lo_image && d.shear_on) {
            // sheared forward, first pass: a = 0 (level 0 has one slope)
            const int p_first = A_off + sg * i0;
            const int X = (sg > 0 ? p_first : p_first - (kV - 1)) - splus;
            // ascending columns of the whole warp item: [Xw0, Xw1)
            const int Xw0 = sg > 0 ? A_off + wbase - splus : A_off - wbase - (32 * kV - 1);
            load_block_a_sheared<SG, RA, Acc, SrcE, NC>(d, S * (1 << M) + s0, X, Xw0,
                                                        Xw0 + 32 * kV, v);
            return;
        }
        if (!d.lo_image && d.lo_win) {
            // windowed level: row s0 + r of group a at its stored index; the
            // 8 columns never wrap inside a window (win_len <= W - 16), and
            // columns outside it feed no stored output, so any in-bounds
            // index (0) serves for them
            const SrcE *base = reinterpret_cast<const SrcE *>(d.lo.ptr);
            const int64_t stride = d.lo.pitch << d.k0;
            const SrcE *p0 = base + ((((int64_t)S << M) + s0) << d.k0) * d.lo.pitch +
                             (int64_t)a * d.lo.pitch;
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int sp = s0 + r;
                const int p_first = A_off + sg * (i0 + a * sp);
                const int lo = sg > 0 ? p_first : p_first - (kV - 1);
                int j = wrap_w(lo - win_base(d, (S << M) + sp, a), d.W);
                if (j >= d.win_len) j = 0;
                load8_fast<SrcE, Acc, NC>(p0 + r * stride, j, v[r]);
                if constexpr (sg < 0) reverse8(v[r]);
            }
            return;
        }
    }
    // ascending source-column range [lo_min, hi_max) over the warp item
    int lo_min, hi_max;
    if (sg > 0) {
        lo_min = A_off + wbase + a * s0;
        hi_max = A_off + wbase + 32 * kV + a * (s0 + RA - 1);
    } else {
        lo_min = A_off - wbase - (32 * kV - 1) - a * (s0 + RA - 1);
        hi_max = A_off - wbase - a * s0 + 1;
    }
    const SrcE *base = reinterpret_cast<const SrcE *>(d.lo.ptr);
    const int row0 = S * (1 << M) + s0;   // first level-0 row (image sources)
    bool interior;
    if (d.lo_image) {
        const int c0 = lo_min - splus, c1 = hi_max - splus;
        if constexpr (ADJ) {
            interior = row0 >= d.src_t_first && row0 + RA - 1 <= d.src_t_last && c0 >= 0 &&
                       c1 <= d.W;
        } else if (d.transpose) {
            interior = c0 >= 0 && c1 <= d.lo.cols && row0 + kV <= d.lo.rows;
        } else {
            interior = c0 >= 0 && c1 <= d.lo.cols && row0 + RA <= d.lo.rows;
        }
    } else {
        interior = lo_min >= 0 && hi_max <= (ADJ ? d.W : d.lo.cols);
    }
    if (!interior) {
        const Block<Acc, RA> b =
            load_block_a_edge<SG, RA, ADJ, Acc, SrcE, NC>(d, M, S, a, s0, A_off, i0);
#pragma unroll
        for (int r = 0; r < RA; ++r)
#pragma unroll
            for (int k = 0; k < kV; ++k) v[r][k] = b.x[r][k];
        return;
    }
    if (!ADJ && d.lo_image && d.transpose) {
        // 8 image rows (buffer columns) x 8 image columns (rows s0..)
        const int p_first = A_off + sg * i0;
        const int lo = (sg > 0 ? p_first : p_first - (kV - 1)) - splus;
        Acc blk[kV][kV];
#pragma unroll
        for (int k = 0; k < kV; ++k)
            load8_fast<SrcE, Acc, NC>(base + (int64_t)(lo + k) * d.lo.pitch, row0, blk[k]);
#pragma unroll
        for (int r = 0; r < RA; ++r)
#pragma unroll
            for (int k = 0; k < kV; ++k) v[r][k] = sg > 0 ? blk[k][r] : blk[kV - 1 - k][r];
        return;
    }
    // row r of the block: one base pointer plus r strides; the column moves by
    // sg*a per row (the shear) for intermediate levels
    int64_t first_row, stride;
    int lo0, dlo;
    {
        const int p_first = A_off + sg * (i0 + a * s0);
        lo0 = sg > 0 ? p_first : p_first - (kV - 1);
        if (d.lo_image) {
            lo0 -= splus;
            dlo = 0;
            if constexpr (ADJ) {
                first_row = (int64_t)d.src_row_base + (int64_t)d.src_row_dir * row0;
                stride = (int64_t)d.src_row_dir * d.lo.pitch;
            } else {
                first_row = row0;
                stride = d.lo.pitch;
            }
        } else {
            first_row = ((int64_t)(S * (1 << M) + s0) << d.k0) + a;
            stride = d.lo.pitch << d.k0;
            dlo = sg * a;
        }
    }
    const SrcE *p0 = base + first_row * d.lo.pitch;
    // Rows that are not sheared against each other (an image's rows) and
    // start on a vector granule, with a row stride of whole granules (a first
    // pass over an aligned image: tiles start on multiples of 8 columns):
    // whole vectors, no realignment. The same for every lane (lanes are 8
    // columns apart), so the branch is warp-uniform.
    // Not compiled for uint16 sources: those are always sheared intermediate
    // levels, whose kernels would only carry the extra code.
    if constexpr (sizeof(SrcE) != 2) {
        constexpr uintptr_t kGran = sizeof(SrcE) == 1 ? 8 : 16;
        if (dlo == 0 && ((reinterpret_cast<uintptr_t>(p0 + lo0) |
                          (uintptr_t)(stride * (int64_t)sizeof(SrcE))) & (kGran - 1)) == 0) {
            const SrcE *p = p0 + lo0;
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                load8_aligned<SrcE, Acc, NC>(p + r * stride, v[r]);
                if constexpr (sg < 0) reverse8(v[r]);
            }
            return;
        }
    }
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        load8_fast<SrcE, Acc, NC>(p0 + r * stride, lo0 + r * dlo, v[r]);
        if constexpr (sg < 0) reverse8(v[r]);
    }
}

// Destination of one lane's 8 buffer columns (i0..i0+7): everything that does
// not depend on the row is computed once per item.
struct DestCols {
    int lo;       // lowest destination column p of the 8
    int X0;       // final level without fhtshift: output column of p = lo
    bool vec;     // the 8 land contiguously, in bounds and 16-byte aligned
};

template <int SG, int FIN, typename Acc, typename DstE>
__device__ __forceinline__ DestCols dest_cols(const PassDesc &d, int D, int i0) {
    DestCols c;
    constexpr int sg = SG;
    const int p_first = D + sg * i0;
    c.lo = sg > 0 ? p_first : p_first - (kV - 1);
    if constexpr (!FIN) {
        c.X0 = c.lo;
        c.vec = c.lo >= 0 && c.lo + kV <= d.hi.cols && (d.hi.pitch & 7) == 0 &&
                (c.lo & 7) == 0 && ((reinterpret_cast<uintptr_t>(d.hi.ptr) & 15) == 0);
        return c;
    } else {
    // column of p: X = p - sigma_plus*n (mod W); fhtshift handled per row
    int X0 = c.lo - (sg > 0 ? d.n : 0);
    if (X0 < 0) X0 += d.W;
    c.X0 = X0;
    c.vec = !d.shift_on && c.lo >= 0 && c.lo + kV <= d.W && X0 + kV <= d.W && (X0 & 3) == 0 &&
            (d.hi.pitch & 3) == 0 && ((reinterpret_cast<uintptr_t>(d.hi.ptr) & 15) == 0);
    return c;
    }
}

// Final-level store of 8 ascending columns p = lo.. of slope t when they do not
// land as one aligned run: cyclic wrap of X, fhtshift rotation, tile borders.
template <typename Acc, typename DstE>
__device__ __noinline__ void store_final_edge(const PassDesc &d, DstE *row, int t, int lo,
                                              Vec8<Acc> v) {
    const int W = d.W, sg = d.sigma;
    int off = sg > 0 ? -d.n : 0;
    if (d.shift_on) {
        const int s = fhtshift_amount(t, W, d.shift_win, sg);
        off += d.shift_inverse ? -s : s;
    }
    off %= W;
    if (off < 0) off += W;
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int p = lo + k;
        if (p >= 0 && p < W) {
            int X = p + off;
            if (X >= W) X -= W;
            if (FHT_STORE_OK(row + X, sizeof(DstE))) row[X] = (DstE)v.x[k];
        }
    }
}

// Store R consecutive level-k1 rows hi_r0.. of this lane's 8 columns: one base
// pointer plus a stride per row; for the final level the rows outside
// [t_first, t_last] (range / full-image maps) are skipped.
template <int SG, int FIN, int R, typename Acc, typename DstE>
__device__ __forceinline__ void store_rows(const PassDesc &d, const DestCols &c, int hi_r0,
                                           const Acc (&v)[R][kV]) {
    DstE *base = reinterpret_cast<DstE *>(d.hi.ptr);
    if constexpr (!FIN) {
        DstE *row = base + (int64_t)hi_r0 * d.hi.pitch;
        const int64_t stride = d.hi.pitch;
        if (c.vec) {   // aligned and in bounds for every row: no per-row checks
            DstE *p = row + c.lo;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                Acc asc[kV];
#pragma unroll
                for (int k = 0; k < kV; ++k) asc[k] = SG > 0 ? v[r][k] : v[r][kV - 1 - k];
                store8_vec<DstE, Acc>(p + r * stride, asc);
            }
            return;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Acc asc[kV];
#pragma unroll
            for (int k = 0; k < kV; ++k) asc[k] = SG > 0 ? v[r][k] : v[r][kV - 1 - k];
            store8<DstE, Acc>(row + r * stride, c.lo, d.hi.cols, asc);
        }
        return;
    } else {
    const int t0 = hi_r0;
    const int r_lo = d.t_first - t0, r_hi = d.t_last - t0;   // rows r in [r_lo, r_hi] exist
    DstE *row = base + ((int64_t)d.row_base + (int64_t)d.row_dir * t0) * d.hi.pitch;
    const int64_t stride = (int64_t)d.row_dir * d.hi.pitch;
    if (c.vec) {   // aligned and in bounds for every row: no per-row checks
        DstE *p = row + c.X0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < r_lo || r > r_hi) continue;
            Acc asc[kV];
#pragma unroll
            for (int k = 0; k < kV; ++k) asc[k] = SG > 0 ? v[r][k] : v[r][kV - 1 - k];
            store8_vec<DstE, Acc, true>(p + r * stride, asc);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < r_lo || r > r_hi) continue;
        Acc asc[kV];
#pragma unroll
        for (int k = 0; k < kV; ++k) asc[k] = SG > 0 ? v[r][k] : v[r][kV - 1 - k];
        {
            Vec8<Acc> e;
#pragma unroll
            for (int k = 0; k < kV; ++k) e.x[k] = asc[k];
            store_final_edge<Acc, DstE>(d, row + r * stride, t0 + r, c.lo, e);
        }
    }
    }
}

// One row of a windowed adjoint level where the lane's 8 columns do not land
// as one run inside the window: each column x < W goes to j = (x - b) mod W
// if j < L.
template <typename Acc, typename DstE>
__device__ __noinline__ void store_win_edge(DstE *row, int lo, int b, int W, int L, Vec8<Acc> v) {
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int x = lo + k;
        if (x >= W) continue;
        int j = x - b;
        if (j < 0) j += W;
        if (j < L && FHT_STORE_OK(row + j, sizeof(DstE))) row[j] = (DstE)v.x[k];
    }
}

// R consecutive rows hi_r0.. of a windowed adjoint level (written by the pass
// before an adjoint's final pass, levels k1): this lane's 8 ascending
// columns lo.. go to each row's window only.
template <int SG, int R, typename Acc, typename DstE>
__device__ __forceinline__ void store_rows_win(const PassDesc &d, int k1, int lo, int hi_r0,
                                               const Acc (&v)[R][kV]) {
    const int W = d.W, L = d.win_len;
    if (lo >= W) return;   // past the level's last column
    DstE *base = reinterpret_cast<DstE *>(d.hi.ptr);
    const int mask = (1 << k1) - 1;
    const bool whole = lo + kV <= W;
    // The R rows are consecutive slopes of one strip s: their windows start
    // sigma*s apart. x is row r's unrounded start, win_c + sigma*(a + r)*s - 8
    // (mod W), advanced by one add and one wrap per row (s < W).
    const int s = hi_r0 >> k1;
    int x = win_base_raw(d, s, hi_r0 & mask);
    // lo and every window start are multiples of 8: with W one too, a row's
    // 8 columns inside its window are one aligned vector
    const bool vec_ok = (W & 7) == 0 && ((d.hi.pitch * (int64_t)sizeof(DstE)) & 15) == 0 &&
                        (reinterpret_cast<uintptr_t>(base) & 15) == 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r > 0) {
            if constexpr (SG > 0) {
                x += s;
                if (x >= W) x -= W;
            } else {
                x -= s;
                if (x < 0) x += W;
            }
        }
        const int row = hi_r0 + r;
        const int b = x & ~7;
        int j = lo - b;
        if (j < 0) j += W;
        if (whole && j >= L && j + kV <= W) continue;   // all 8 outside the window
        Acc asc[kV];
#pragma unroll
        for (int k = 0; k < kV; ++k) asc[k] = SG > 0 ? v[r][k] : v[r][kV - 1 - k];
        DstE *rp = base + (int64_t)row * d.hi.pitch;
        if (whole && j + kV <= L) {
            if (vec_ok) store8_vec<DstE, Acc>(rp + j, asc);
            else store8<DstE, Acc>(rp, j, L, asc);
        } else {
            Vec8<Acc> e;
#pragma unroll
            for (int k = 0; k < kV; ++k) e.x[k] = asc[k];
            store_win_edge<Acc, DstE>(rp, lo, b, W, L, e);
        }
    }
}

// Does any of the R rows hi_r0.. of a windowed adjoint level take a column
// of [xa, xa + len)? (warp-uniform: decides whether a block-B item runs)
template <int R>
__device__ __forceinline__ bool win_rows_hit(const PassDesc &d, int k1, int hi_r0, int xa,
                                             int len) {
    const int W = d.W, L = d.win_len, mask = (1 << k1) - 1;
    if (xa >= W) return false;
    if (len > W - xa) len = W - xa;
    bool hit = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = hi_r0 + r;
        int j = xa - win_base(d, row >> k1, row & mask);
        if (j < 0) j += W;
        hit |= j < L || j + len > W;
    }
    return hit;
}

// Final level of an adjoint: R consecutive output rows y0.. (image rows of the
// (transposed) image) x this lane's 8 columns go to the image gradient,
// cropped to dst_h x dst_w, transposed for the horizontal quadrants, added to
// the gradient already there when accumulating.
template <typename E, typename Acc>
__device__ __forceinline__ E acc_store(E old, Acc v, bool acc) {
    return acc ? (E)Arith<Acc>::add((Acc)old, v) : (E)v;
}

// Out-of-line fallbacks of store_image_block (crop edges, unaligned rows).
// One image row: the lane's 8 ascending columns p = lo.. at X0.., those with
// p in [p_lo, p_hi) only.
template <typename Acc, typename DstE>
__device__ __noinline__ void store_image_row_edge(DstE *row, int X0, int lo, int p_lo, int p_hi,
                                                  int acc, Vec8<Acc> a) {
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int p = lo + k;
        if (p >= p_lo && p < p_hi && FHT_STORE_OK(row + X0 + k, sizeof(DstE)))
            row[X0 + k] = acc_store<DstE, Acc>(row[X0 + k], a.x[k], acc);
    }
}

// One image row X of a transposed destination: columns y0..y0+R-1 (< dst_h).
template <int R, typename Acc, typename DstE>
__device__ __noinline__ void store_image_col_edge(DstE *row, int y0, int dst_h, int acc,
                                                  Vec8<Acc> col) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = y0 + r;
        if (y < dst_h && FHT_STORE_OK(row + y, sizeof(DstE)))
            row[y] = acc_store<DstE, Acc>(row[y], col.x[r], acc);
    }
}

// Final level of an adjoint: R consecutive output rows y0.. x this lane's 8
// columns go to the image gradient, cropped to dst_h x dst_w, transposed for
// the horizontal quadrants (TR), added to the gradient already there when
// accumulating. Columns p in [p_begin, p_begin + p_count) are exactly the
// image columns X = p - sigma_plus*n < dst_w (a tile wider than W would
// otherwise reach the same X again through the cyclic wrap). When
// accumulating, the old values of up to 4 rows (columns) are loaded before
// any of their sums is stored, so those loads are in flight together.
template <int SG, bool TR, int R, typename Acc, typename DstE>
__device__ __forceinline__ void store_image_block(const PassDesc &d, int y0, int lo,
                                                  const Acc (&v)[R][kV]) {
    constexpr int sg = SG;
    constexpr int kB = 4;   // rows (columns) whose old values are loaded together
    const int acc = d.accumulate;
    const int p_lo = d.p_begin, p_hi = d.p_begin + d.p_count;
    const int X0 = lo - (sg > 0 ? d.n : 0);   // column of p = lo (valid when lo >= p_lo)
    DstE *img = reinterpret_cast<DstE *>(d.hi.ptr);
    const int64_t pitch = d.hi.pitch;
    const bool inside = lo >= p_lo && lo + kV <= p_hi;
    using V4 = typename std::conditional<std::is_same<DstE, float>::value, float4, int4>::type;
    if constexpr (!TR) {
        const bool vec = inside && (X0 & 3) == 0 && (pitch & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(img) & 15) == 0);
        const int rows = d.dst_h - y0;   // rows r < rows exist
        const int r_lo = d.dst_row_lo - y0;   // ... and rows r >= r_lo
        if (vec) {
            DstE *base = img + (int64_t)(y0 - d.dst_row_lo) * pitch + X0;
            if (!acc) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r >= rows || r < r_lo) continue;
                    if (!FHT_STORE_OK(base + r * pitch, kV * sizeof(DstE))) continue;
                    V4 a, b;
                    a.x = (DstE)v[r][sg > 0 ? 0 : 7];
                    a.y = (DstE)v[r][sg > 0 ? 1 : 6];
                    a.z = (DstE)v[r][sg > 0 ? 2 : 5];
                    a.w = (DstE)v[r][sg > 0 ? 3 : 4];
                    b.x = (DstE)v[r][sg > 0 ? 4 : 3];
                    b.y = (DstE)v[r][sg > 0 ? 5 : 2];
                    b.z = (DstE)v[r][sg > 0 ? 6 : 1];
                    b.w = (DstE)v[r][sg > 0 ? 7 : 0];
                    V4 *q = reinterpret_cast<V4 *>(base + r * pitch);
                    q[0] = a;
                    q[1] = b;
                }
                return;
            }
#pragma unroll
            for (int r0 = 0; r0 < R; r0 += kB) {
                constexpr int B = R < kB ? R : kB;
                V4 old[B][2];
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    if (r0 + j < rows && r0 + j >= r_lo &&
                        FHT_STORE_OK(base + (r0 + j) * pitch, kV * sizeof(DstE))) {
                        const V4 *q = reinterpret_cast<const V4 *>(base + (r0 + j) * pitch);
                        old[j][0] = q[0];
                        old[j][1] = q[1];
                    }
                }
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    const int r = r0 + j;
                    if (r >= rows || r < r_lo) continue;
                    if (!FHT_STORE_OK(base + r * pitch, kV * sizeof(DstE))) continue;
                    Acc asc[kV];
#pragma unroll
                    for (int k = 0; k < kV; ++k) asc[k] = sg > 0 ? v[r][k] : v[r][kV - 1 - k];
                    V4 a, b;
                    a.x = (DstE)Arith<Acc>::add((Acc)old[j][0].x, asc[0]);
                    a.y = (DstE)Arith<Acc>::add((Acc)old[j][0].y, asc[1]);
                    a.z = (DstE)Arith<Acc>::add((Acc)old[j][0].z, asc[2]);
                    a.w = (DstE)Arith<Acc>::add((Acc)old[j][0].w, asc[3]);
                    b.x = (DstE)Arith<Acc>::add((Acc)old[j][1].x, asc[4]);
                    b.y = (DstE)Arith<Acc>::add((Acc)old[j][1].y, asc[5]);
                    b.z = (DstE)Arith<Acc>::add((Acc)old[j][1].z, asc[6]);
                    b.w = (DstE)Arith<Acc>::add((Acc)old[j][1].w, asc[7]);
                    V4 *q = reinterpret_cast<V4 *>(base + r * pitch);
                    q[0] = a;
                    q[1] = b;
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= rows || r < r_lo) continue;
                Vec8<Acc> a;
#pragma unroll
                for (int k = 0; k < kV; ++k) a.x[k] = sg > 0 ? v[r][k] : v[r][kV - 1 - k];
                store_image_row_edge<Acc, DstE>(img + (int64_t)(y0 + r - d.dst_row_lo) * pitch,
                                                X0, lo, p_lo, p_hi, acc, a);
            }
        }
    } else {
        // transposed: column k of the lane's 8 is image row X0 + k, image
        // columns y0 .. y0 + R - 1
        bool vec = false;
        if constexpr (R >= 4) {
            vec = inside && y0 + R <= d.dst_h && (pitch & 3) == 0 &&
                  ((reinterpret_cast<uintptr_t>(img + y0) & 15) == 0);
        }
        if (vec) {
            constexpr int NV = R / 4 > 0 ? R / 4 : 1;   // 16-byte vectors per column
            if (!acc) {
#pragma unroll
                for (int k = 0; k < kV; ++k) {
                    const int kk = sg > 0 ? k : kV - 1 - k;
                    V4 *q = reinterpret_cast<V4 *>(img + (int64_t)(X0 + k) * pitch + y0);
                    if (!FHT_STORE_OK(q, NV * sizeof(V4))) continue;
#pragma unroll
                    for (int u = 0; u < NV; ++u) {
                        V4 o;
                        o.x = (DstE)v[4 * u + 0][kk];
                        o.y = (DstE)v[4 * u + 1][kk];
                        o.z = (DstE)v[4 * u + 2][kk];
                        o.w = (DstE)v[4 * u + 3][kk];
                        q[u] = o;
                    }
                }
                return;
            }
#pragma unroll
            for (int k0 = 0; k0 < kV; k0 += kB) {
                V4 old[kB][NV];
#pragma unroll
                for (int j = 0; j < kB; ++j)
#pragma unroll
                    for (int u = 0; u < NV; ++u)
                        old[j][u] = FHT_LOAD_OK(img + (int64_t)(X0 + k0 + j) * pitch + y0,
                                                NV * sizeof(V4))
                                        ? reinterpret_cast<const V4 *>(
                                              img + (int64_t)(X0 + k0 + j) * pitch + y0)[u]
                                        : V4{};
#pragma unroll
                for (int j = 0; j < kB; ++j) {
                    const int k = k0 + j;
                    const int kk = sg > 0 ? k : kV - 1 - k;
                    V4 *q = reinterpret_cast<V4 *>(img + (int64_t)(X0 + k) * pitch + y0);
                    if (!FHT_STORE_OK(q, NV * sizeof(V4))) continue;
#pragma unroll
                    for (int u = 0; u < NV; ++u) {
                        V4 o = old[j][u];
                        o.x = (DstE)Arith<Acc>::add((Acc)o.x, v[4 * u + 0][kk]);
                        o.y = (DstE)Arith<Acc>::add((Acc)o.y, v[4 * u + 1][kk]);
                        o.z = (DstE)Arith<Acc>::add((Acc)o.z, v[4 * u + 2][kk]);
                        o.w = (DstE)Arith<Acc>::add((Acc)o.w, v[4 * u + 3][kk]);
                        q[u] = o;
                    }
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < kV; ++k) {
                const int p = lo + k;
                if (p < p_lo || p >= p_hi) continue;
                Vec8<Acc> col;
#pragma unroll
                for (int r = 0; r < kV; ++r)
                    col.x[r] = r < R ? (sg > 0 ? v[r < R ? r : 0][k] : v[r < R ? r : 0][kV - 1 - k])
                                     : Acc(0);
                store_image_col_edge<R, Acc, DstE>(img + (int64_t)(X0 + k) * pitch, y0, d.dst_h,
                                                   acc, col);
            }
        }
    }
}

// Is the whole tile inside the black zone of every slope of the group?
// (final level only: slopes t in [a*2^M, a*2^M + 2^M - 1])
__device__ __forceinline__ bool tile_all_black(const PassDesc &d, int M, int a, int p0,
                                               int tile_out) {
    if (d.cyclic) return false;
    const int t_max = (a << M) + (1 << M) - 1;
    const int lo = p0, hi = p0 + tile_out;   // [lo, hi) in p
    if (d.sigma > 0) {
        // zero for p in [0, n - t) and p in [w_c + n, W)
        return hi <= d.n - t_max || lo >= d.black_wc + d.n;
    }
    // sigma = -1: zero for p in [w_c + t, W)
    return lo >= d.black_wc + t_max;
}

// Sheared forward, first pass: is the tile [p0, p0 + T) outside the content of
// its strip S? The strip's image rows y (level k1 = M) are rotated by s(y),
// monotone in y, so its level-k1 rows are zero outside the columns
// [s_lo, s_hi + w + 2^k1] (cyclic; both signs' compact columns fall inside).
__device__ __forceinline__ bool sheared_tile_zero(const PassDesc &d, int M, int S, int p0,
                                                  int T) {
    const int y0 = S << M;
    int y1 = y0 + (1 << M) - 1;
    if (y1 >= d.lo.rows) y1 = d.lo.rows - 1;
    if (y1 < y0) return true;   // no image row in the strip
    const int sa = shear_shift(d, y0), sb = shear_shift(d, y1);
    const int lo = sa < sb ? sa : sb, hi = sa < sb ? sb : sa;
    const int len = hi - lo + d.lo.cols + (1 << M) + 1;
    if (len + T >= d.W) return false;
    const int j = wrap_w(p0 - lo, d.W);
    return !(j < len || j + T > d.W);
}

// Windowed adjoint level: may any of the 2^M rows of group (S, a) keep a
// column of the tile [p0, p0 + T)? Row (S, a*2^M + c) keeps the window of
// win_len columns from about win_c + sigma*(a*2^M + c)*S (win_base, 8 to 15
// columns earlier, on a multiple of 8), so over c the windows form one
// cyclic arc (consecutive windows start S <= win_len apart) from
// win_c - 15 + sigma*a*2^M*S + min(0, sigma*(2^M - 1)*S), of length at most
// win_len + (2^M - 1)*S + 15. A tile outside that arc is never read by the
// final pass and is skipped whole. (Conservative: a tile the arc only
// grazes still runs.) For small S the arc is little more than one window, so
// most tiles of the row are skipped.
__device__ __forceinline__ bool group_window_hit(const PassDesc &d, int M, int S, int a, int p0,
                                                 int T) {
    const int W = d.W;
    if (p0 >= W) return false;
    const int len = T < W - p0 ? T : W - p0;
    const long long spread = (long long)((1 << M) - 1) * S;
    const long long span = d.win_len + spread + 16;
    if (span + len >= W) return true;
    long long start = (long long)d.win_c - 16 + (long long)d.sigma * a * (1 << M) * S;
    if (d.sigma < 0) start -= spread;
    int j = (int)(((long long)p0 - start) % W);
    if (j < 0) j += W;
    return j < span || j + len > W;
}

// Where one (group, tile) item of a pass sits: its group (S, a), first
// output column p0, the buffer column offsets of its source (A_off) and
// destination (D), and whether the whole tile is black (all zero).
struct ItemPos {
    int S, a, p0, A_off, D;
    bool black;
};

template <int M, int SG, bool ADJ, int FIN>
__device__ __forceinline__ ItemPos item_pos(const PassDesc &d, int T, int gy, int tile) {
    ItemPos ip;
    ip.S = gy / d.a_count;
    ip.a = d.a_lo + gy % d.a_count;
    ip.p0 = d.p_begin + tile * T;
    ip.A_off = SG > 0 ? ip.p0 - (1 << (d.k0 + M)) + (1 << d.k0) : ip.p0 + T - 1;
    ip.D = SG > 0 ? ip.p0 : ip.p0 + T - 1;
    if constexpr (ADJ && !FIN)
        ip.black = (d.shear_on && d.lo_image && sheared_tile_zero(d, M, ip.S, ip.p0, T)) ||
                   (d.hi_win && !group_window_hit(d, M, ip.S, ip.a, ip.p0, T));
    else
        ip.black = !ADJ && FIN && tile_all_black(d, M, ip.a, ip.p0, T);
    return ip;
}

// Block A of a two-block item (MB > 0): warps warp, warp + nwarps, ... load
// mini-strips of RA source rows, run MA levels in registers and write the
// results to the shared tile sm (nothing to do for a black tile).
template <int MA, int MB, int SG, bool ADJ, typename Acc, typename SrcE, typename MidE,
          int OP = 0, bool NC = true>
__device__ __forceinline__ void tile_block_a(const PassDesc &d, const TileGeom &G,
                                             const ItemPos &ip, MidE *sm, int warp, int nwarps,
                                             int lane) {
    constexpr int M = MA + MB, RA = 1 << MA, RB = 1 << MB;
    constexpr int PAD = TilePad<MidE>::kPad;
    const int P = G.pitch;
    if (ip.black) return;
    // mini-strip g (rows g*RA + rho), warp-column wc
    for (int item = warp; item < RB * G.n_a; item += nwarps) {
        const int g = item % RB, wc = item / RB;
        const int i0 = wc * kWarpValid + lane * kV;
        Acc v[RA][kV];
        load_block_a<SG, RA, ADJ, Acc, SrcE, NC>(d, M, ip.S, ip.a, g * RA, ip.A_off,
                                                 wc * kWarpValid, i0, v);
        reg_butterfly<MA, Acc, OP>(v);
        if (lane < kLanesValid) {
            const int pos = (8 + PAD) * (i0 >> 3);   // i0 is a multiple of 8
#pragma unroll
            for (int c = 0; c < RA; ++c) {
                MidE *row = sm + (g * RA + c) * P + pos;
                if constexpr (PAD == 2) {
                    uint32_t *w = reinterpret_cast<uint32_t *>(row);
#pragma unroll
                    for (int k = 0; k < kV / 2; ++k)
                        w[k] = pack_u16x2((uint32_t)v[c][2 * k], (uint32_t)v[c][2 * k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < kV; ++k) row[k] = (MidE)v[c][k];
                }
            }
        }
    }
}

// Transposed image gradient (an adjoint's final pass for Q2/Q3) through
// shared memory. Block B's item a2 holds, per lane, 8 image rows X (its
// buffer columns) x RB image columns y (its output rows); stored straight, a
// warp's 16-byte pieces land in 32 different image rows. Instead, every warp
// writes its values into the tile region as [xi][y] rows of 2^M floats
// (xi = X - X_base < T, y - y_base < 2^M), 16-byte granules XOR-swizzled by
// (xi >> 3) so that neither the writes (lanes 8 rows apart) nor the reads
// (consecutive granules of a row) conflict; after a CTA barrier the whole
// CTA adds each image row's 2^M columns as contiguous float4s (old value
// first, as acc_store does). Used when every warp has exactly one block-B
// item (the caller checks), RB >= 4 and the tile region holds T x 2^M values.
template <int M>
__device__ __forceinline__ int stage_granule(int xi, int gi) {
    constexpr int G = (1 << M) / 4;   // granules per staged row
    return xi * G + (gi ^ ((xi >> 3) & (G - 1) & 7));
}

template <int SG, int M, int RB, typename Acc>
__device__ __forceinline__ void stage_transposed(float *st, int T, int i0, int yo0,
                                                 const Acc (&v)[RB][kV]) {
#pragma unroll
    for (int k = 0; k < kV; ++k) {
        const int xi = SG > 0 ? i0 + k : T - 1 - (i0 + k);
#pragma unroll
        for (int h = 0; h < RB / 4; ++h) {
            const float4 q = make_float4((float)v[4 * h][k], (float)v[4 * h + 1][k],
                                         (float)v[4 * h + 2][k], (float)v[4 * h + 3][k]);
            reinterpret_cast<float4 *>(st)[stage_granule<M>(xi, yo0 / 4 + h)] = q;
        }
    }
}

// The CTA's cooperative store of the staged block: image rows X_base + xi
// (xi < T, X < dst_w... the transposed image's column count is dst_w), image
// columns y_base .. y_base + 2^M - 1 (< dst_h), added into the gradient when
// accumulating.
template <int M, typename DstE>
__device__ __forceinline__ void store_staged_transposed(const PassDesc &d, const float *st, int T,
                                                        int X_base, int y_base) {
    constexpr int G = (1 << M) / 4;
    constexpr int kB = 4;   // granules per thread whose old values are loaded together
    DstE *img = reinterpret_cast<DstE *>(d.hi.ptr);
    const int64_t pitch = d.hi.pitch;
    const bool vec = (pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
    const int acc = d.accumulate;
    const int total = T * G, step = blockDim.x;
    for (int base = threadIdx.x; base < total; base += kB * step) {
        float4 q[kB], old[kB];
        DstE *p[kB];
        int mode[kB];   // 0 nothing, 1 vector, 2 scalar
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int idx = base + u * step;
            mode[u] = 0;
            p[u] = img;
            if (idx >= total) continue;
            const int xi = idx / G, gi = idx - xi * G;
            const int X = X_base + xi, y = y_base + 4 * gi;
            if (X < 0 || X >= d.dst_w || y >= d.dst_h) continue;
            q[u] = reinterpret_cast<const float4 *>(st)[stage_granule<M>(xi, gi)];
            p[u] = img + (int64_t)X * pitch + y;
            mode[u] = vec && y + 4 <= d.dst_h ? 1 : 2;
            if (mode[u] == 1 && !FHT_STORE_OK(p[u], sizeof(float4))) mode[u] = 0;
            if (mode[u] == 1 && acc) old[u] = *reinterpret_cast<const float4 *>(p[u]);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (mode[u] == 1) {
                float4 o = q[u];
                if (acc) {
                    o.x = __fadd_rn(old[u].x, q[u].x);
                    o.y = __fadd_rn(old[u].y, q[u].y);
                    o.z = __fadd_rn(old[u].z, q[u].z);
                    o.w = __fadd_rn(old[u].w, q[u].w);
                }
                *reinterpret_cast<float4 *>(p[u]) = o;
            } else if (mode[u] == 2) {
                const int y0 = (int)((p[u] - img) % pitch);
                const float e[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (y0 + c < d.dst_h && FHT_STORE_OK(p[u] + c, sizeof(DstE)))
                        p[u][c] = acc ? __fadd_rn((float)p[u][c], e[c]) : e[c];
            }
        }
    }
}

// Block B of a two-block item: level-MA slope a2 of every mini-strip g, read
// from the shared tile with the shear a2*g, MB more levels, then the
// destination (zeros for a black tile, without reading the tile).
template <int MA, int MB, int SG, bool ADJ, int FIN, typename Acc, typename MidE, typename DstE,
          int OP = 0>
__device__ __forceinline__ void tile_block_b(const PassDesc &d, const TileGeom &G,
                                             const ItemPos &ip, const MidE *sm, int warp,
                                             int nwarps, int lane) {
    constexpr int M = MA + MB, RA = 1 << MA, RB = 1 << MB;
    constexpr int PAD = TilePad<MidE>::kPad;
    const int P = G.pitch, T = G.tile_out;
    // an adjoint's transposed image gradient through the tile region (see
    // stage_transposed): every warp one item, all items barriered together
    constexpr bool kStageTr = ADJ && FIN == 2 && RB >= 4 && std::is_same<DstE, float>::value &&
                              std::is_same<Acc, float>::value;
    if constexpr (kStageTr) {
        if (RA * G.n_b == nwarps) {
            const int a2 = warp;
            const int slope0 = (ip.a << M) + a2 * RB;
            const bool run = !(slope0 > d.need_hi || slope0 + RB - 1 < d.need_lo);
            const int i0 = lane * kV;
            const int i0r = i0 < T ? i0 : T;
            Acc v[RB][kV];
            if (run) {
#pragma unroll
                for (int g = 0; g < RB; ++g) {
                    const int x0 = i0r + a2 * g;
                    const int delta = x0 & 7;
                    const MidE *row = sm + (g * RA + a2) * P + tile_pos(x0, PAD);
                    MidE raw[kV + PAD];
#pragma unroll
                    for (int j = 0; j < kV + PAD; ++j) raw[j] = row[j];
#pragma unroll
                    for (int k = 0; k < kV; ++k)
                        v[g][k] = (Acc)(k + delta >= kV ? raw[k + PAD] : raw[k]);
                }
                reg_butterfly<MB, Acc, OP>(v);
            }
            __syncthreads();   // every warp has read the tile: it becomes the staging area
            float *st = reinterpret_cast<float *>(const_cast<MidE *>(sm));
            if (run && lane < kLanesValid && i0 < T)
                stage_transposed<SG, M, RB, Acc>(st, T, i0, a2 * RB, v);
            __syncthreads();
            // buffer column i = 0 is p = D (sign +) or D - (T - 1) (sign -); X = p - sigma_plus*n
            const int p_lo_tile = SG > 0 ? ip.D : ip.D - (T - 1);
            const int X_base = p_lo_tile - (SG > 0 ? d.n : 0);
            store_staged_transposed<M, DstE>(d, st, T, X_base, hi_row(d, M, ip.S, ip.a, 0));
            return;
        }
    }
    for (int item = warp; item < RA * G.n_b; item += nwarps) {
        const int a2 = item % RA, jc = item / RA;
        // level-k1 slopes (a << M) + a2*RB .. + RB - 1 of this item: skip it
        // when none is used later
        const int slope0 = (ip.a << M) + a2 * RB;
        if (slope0 > d.need_hi || slope0 + RB - 1 < d.need_lo) continue;
        if constexpr (ADJ && !FIN) {
            // windowed level: skip the item when no row's window meets the
            // warp's columns
            if (d.hi_win) {
                const int c0 = jc * kWarpValid;
                const int cnt = T - c0 < kWarpValid ? T - c0 : kWarpValid;
                const int xa = SG > 0 ? ip.D + c0 : ip.D - c0 - cnt + 1;
                if (!win_rows_hit<RB>(d, d.k0 + M, hi_row(d, M, ip.S, ip.a, a2 * RB), xa, cnt))
                    continue;
            }
        }
        const int i0 = jc * kWarpValid + lane * kV;
        // lanes past the tile store nothing: they read where the first of
        // them reads, so the tile ends where that lane's columns end
        const int i0r = i0 < T ? i0 : T;
        Acc v[RB][kV];
        if (!ip.black) {
#pragma unroll
            for (int g = 0; g < RB; ++g) {
                const int x0 = i0r + a2 * g;
                const int delta = x0 & 7;
                const MidE *row = sm + (g * RA + a2) * P + tile_pos(x0, PAD);
                MidE raw[kV + PAD];
#pragma unroll
                for (int j = 0; j < kV + PAD; ++j) raw[j] = row[j];
#pragma unroll
                for (int k = 0; k < kV; ++k)
                    v[g][k] = (Acc)(k + delta >= kV ? raw[k + PAD] : raw[k]);
            }
            reg_butterfly<MB, Acc, OP>(v);
        } else {
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int k = 0; k < kV; ++k) v[r][k] = Acc(0);
        }
        if (lane < kLanesValid && i0 < T) {
            const DestCols dc = dest_cols<SG, FIN, Acc, DstE>(d, ip.D, i0);
            if constexpr (ADJ && FIN) {
                store_image_block<SG, FIN == 2, RB, Acc, DstE>(d, hi_row(d, M, ip.S, ip.a, a2 * RB), dc.lo,
                                                     v);
            } else if (ADJ && !FIN && d.hi_win) {
                store_rows_win<SG, RB, Acc, DstE>(d, d.k0 + M, dc.lo,
                                                  hi_row(d, M, ip.S, ip.a, a2 * RB), v);
            } else {
                store_rows<SG, FIN, RB, Acc, DstE>(d, dc, hi_row(d, M, ip.S, ip.a, a2 * RB), v);
            }
        }
    }
}

// ------------------------------------------------------------ packed first pass

// Block A's RA rows of a uint8 image as packed words in buffer order: an
// aligned interior item reads one 8-byte vector per row and packs its bytes
// straight into 16-bit halves; every other case (image edges, unaligned rows,
// the transposed load) takes the general loader and packs its values.
template <int SG, int RA>
__device__ __forceinline__ void load_block_a_u8x2(const PassDesc &d, int M, int S, int s0,
                                                  int A_off, int wbase, int i0,
                                                  uint32_t (&w)[RA][4]) {
    constexpr int sg = SG;
    const int splus = sg > 0 ? 1 : 0;
    if (!d.transpose) {
        const int lo_min = sg > 0 ? A_off + wbase : A_off - wbase - (32 * kV - 1);
        const int hi_max = sg > 0 ? A_off + wbase + 32 * kV : A_off - wbase + 1;
        const int row0 = S * (1 << M) + s0;
        const int p_first = A_off + sg * i0;
        const int lo0 = (sg > 0 ? p_first : p_first - (kV - 1)) - splus;
        const uint8_t *p = reinterpret_cast<const uint8_t *>(d.lo.ptr) + (int64_t)row0 * d.lo.pitch + lo0;
        if (lo_min - splus >= 0 && hi_max - splus <= d.lo.cols && row0 + RA <= d.lo.rows &&
            ((reinterpret_cast<uintptr_t>(p) | (uintptr_t)d.lo.pitch) & 7) == 0) {
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const uint8_t *q8 = p + (int64_t)r * d.lo.pitch;
                uint2 q = make_uint2(0u, 0u);
                if (FHT_LOAD_OK(q8, 8)) q = ldvec<true>(reinterpret_cast<const uint2 *>(q8));
                if constexpr (sg > 0) {
                    w[r][0] = __byte_perm(q.x, 0u, 0x4140u);
                    w[r][1] = __byte_perm(q.x, 0u, 0x4342u);
                    w[r][2] = __byte_perm(q.y, 0u, 0x4140u);
                    w[r][3] = __byte_perm(q.y, 0u, 0x4342u);
                } else {   // buffer order runs down the image columns
                    w[r][0] = __byte_perm(q.y, 0u, 0x4243u);
                    w[r][1] = __byte_perm(q.y, 0u, 0x4041u);
                    w[r][2] = __byte_perm(q.x, 0u, 0x4243u);
                    w[r][3] = __byte_perm(q.x, 0u, 0x4041u);
                }
            }
            return;
        }
    }
    int32_t v[RA][kV];
    load_block_a<SG, RA, false, int32_t, uint8_t>(d, M, S, 0, s0, A_off, wbase, i0, v);
#pragma unroll
    for (int r = 0; r < RA; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) w[r][j] = pack_u16x2((uint32_t)v[r][2 * j], (uint32_t)v[r][2 * j + 1]);
}

// Word j of 8 buffer columns from x0 of a uint16 tile row (the two 8-column
// groups around x0, with the pad word between them skipped).
__device__ __forceinline__ void tile_read_u16x2(const uint16_t *row_group, int delta,
                                                uint32_t (&w)[4]) {
    const uint32_t *g = reinterpret_cast<const uint32_t *>(row_group);
    // words of the two groups without the pad: e[0..3] group A, e[4..7] group B
    uint32_t e[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        e[i] = g[i];
        e[4 + i] = g[5 + i];
    }
    const int m = delta >> 1;
    uint32_t u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
        u[i] = sel4(e[i], e[i + 1 < 8 ? i + 1 : 7], e[i + 2 < 8 ? i + 2 : 7],
                    e[i + 3 < 8 ? i + 3 : 7], m);
    if (delta & 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = __byte_perm(u[j], u[j + 1], 0x5432u);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = u[j];
    }
}

// The two-block first pass of a sum transform from a uint8 image into a
// uint16 level, on packed words (the generic item's steps, same results).
template <int MA, int MB, int SG>
__device__ void packed_first_item(const PassDesc &d, int gy, int tile, uint16_t *sm) {
    constexpr int M = MA + MB, RA = 1 << MA, RB = 1 << MB, PAD = 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const TileGeom G = tile_geom(MA, MB, d.n_a, nwarps, PAD);
    const int T = G.tile_out, P = G.pitch;
    const ItemPos ip = item_pos<M, SG, false, 0>(d, T, gy, tile);
    // block A: image rows -> MA levels -> shared tile (packed words)
    for (int item = warp; item < RB * G.n_a; item += nwarps) {
        const int g = item % RB, wc = item / RB;
        const int i0 = wc * kWarpValid + lane * kV;
        uint32_t w[RA][4];
        load_block_a_u8x2<SG, RA>(d, M, ip.S, g * RA, ip.A_off, wc * kWarpValid, i0, w);
        reg_butterfly_u16x2<MA>(w);
        if (lane < kLanesValid) {
            const int pos = (8 + PAD) * (i0 >> 3);
#pragma unroll
            for (int c = 0; c < RA; ++c) {
                uint32_t *row = reinterpret_cast<uint32_t *>(sm + (g * RA + c) * P + pos);
#pragma unroll
                for (int j = 0; j < 4; ++j) row[j] = w[c][j];
            }
        }
    }
    __syncthreads();
    // block B: level-MA slope a2 of every mini-strip -> MB levels -> the level
    for (int item = warp; item < RA * G.n_b; item += nwarps) {
        const int a2 = item % RA, jc = item / RA;
        const int slope0 = (ip.a << M) + a2 * RB;
        if (slope0 > d.need_hi || slope0 + RB - 1 < d.need_lo) continue;
        const int i0 = jc * kWarpValid + lane * kV;
        const int i0r = i0 < T ? i0 : T;
        uint32_t w[RB][4];
#pragma unroll
        for (int g = 0; g < RB; ++g) {
            const int x0 = i0r + a2 * g;
            tile_read_u16x2(sm + (g * RA + a2) * P + tile_pos(x0 & ~7, PAD), x0 & 7, w[g]);
        }
        reg_butterfly_u16x2<MB>(w);
        if (lane < kLanesValid && i0 < T) {
            const DestCols dc = dest_cols<SG, 0, int32_t, uint16_t>(d, ip.D, i0);
            uint16_t *row = reinterpret_cast<uint16_t *>(d.hi.ptr) +
                            (int64_t)hi_row(d, M, ip.S, ip.a, a2 * RB) * d.hi.pitch;
            if (dc.vec) {
                uint16_t *p = row + dc.lo;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    uint4 q;
                    if constexpr (SG > 0) {
                        q = make_uint4(w[r][0], w[r][1], w[r][2], w[r][3]);
                    } else {   // ascending columns: words and halves reversed
                        q = make_uint4(__byte_perm(w[r][3], 0u, 0x1032u),
                                       __byte_perm(w[r][2], 0u, 0x1032u),
                                       __byte_perm(w[r][1], 0u, 0x1032u),
                                       __byte_perm(w[r][0], 0u, 0x1032u));
                    }
                    uint16_t *pr = p + (int64_t)r * d.hi.pitch;
                    if (FHT_STORE_OK(pr, 16)) *reinterpret_cast<uint4 *>(pr) = q;
                }
            } else {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    int32_t asc[kV];
#pragma unroll
                    for (int k = 0; k < kV; ++k) {
                        const int kb = SG > 0 ? k : kV - 1 - k;   // buffer column
                        asc[k] = (int32_t)((w[r][kb >> 1] >> (16 * (kb & 1))) & 0xffffu);
                    }
                    store8<uint16_t, int32_t>(row + (int64_t)r * d.hi.pitch, dc.lo, d.hi.cols, asc);
                }
            }
        }
    }
}

// One item with all the CTA's warps: single register block (MB = 0), or
// block A, a CTA barrier, block B.
// ADJ selects the adjoint form at compile time (cyclic columns, row-mapped
// gradient source, image-gradient destination) so the forward kernels carry
// none of its code; FIN likewise selects the destination (0 an intermediate
// level, 1 the caller's layout, 2 an adjoint's transposed image gradient), so
// each kernel holds one store path. OP is the operation along the patterns
// (Combine: 0 the sum, 1 the maximum, 2 the minimum). NC = false reads the
// source through coherent loads (a level written earlier in the same launch;
// see ldvec).
template <int MA, int MB, int SG, bool ADJ, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE, int OP = 0, bool NC = true>
__device__ void fused_forward_item(const PassDesc &d, int gy, int tile, MidE *sm) {
    constexpr int M = MA + MB, RA = 1 << MA;
    constexpr int PAD = TilePad<MidE>::kPad;
    FHT_DEBUG_BEGIN(d);
    // the first pass of a sum over a uint8 image into a uint16 level: packed
    // (its source is the caller's image, read-only in any launch)
    if constexpr (!ADJ && FIN == 0 && OP == 0 && MB > 0 &&
                  std::is_same<Acc, int32_t>::value && std::is_same<SrcE, uint8_t>::value &&
                  std::is_same<MidE, uint16_t>::value && std::is_same<DstE, uint16_t>::value) {
        packed_first_item<MA, MB, SG>(d, gy, tile, sm);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const TileGeom G = tile_geom(MA, MB, d.n_a, nwarps, PAD);
    const int T = G.tile_out;
    const ItemPos ip = item_pos<M, SG, ADJ, FIN>(d, T, gy, tile);

    if constexpr (MB == 0) {
        // single register block: source -> registers -> destination
        for (int item = warp; item < G.n_a; item += nwarps) {
            const int i0 = item * kWarpValid + lane * kV;
            Acc v[RA][kV];
            if (!ip.black) {
                load_block_a<SG, RA, ADJ, Acc, SrcE, NC>(d, M, ip.S, ip.a, 0, ip.A_off,
                                                         item * kWarpValid, i0, v);
                reg_butterfly<MA, Acc, OP>(v);
            } else {
#pragma unroll
                for (int r = 0; r < RA; ++r)
#pragma unroll
                    for (int k = 0; k < kV; ++k) v[r][k] = Acc(0);
            }
            if (lane < kLanesValid && i0 < T) {
                const DestCols dc = dest_cols<SG, FIN, Acc, DstE>(d, ip.D, i0);
                if constexpr (ADJ && FIN) {
                    store_image_block<SG, FIN == 2, RA, Acc, DstE>(d, hi_row(d, M, ip.S, ip.a, 0), dc.lo, v);
                } else if (ADJ && !FIN && d.hi_win) {
                    store_rows_win<SG, RA, Acc, DstE>(d, d.k0 + M, dc.lo,
                                                      hi_row(d, M, ip.S, ip.a, 0), v);
                } else {
                    store_rows<SG, FIN, RA, Acc, DstE>(d, dc, hi_row(d, M, ip.S, ip.a, 0), v);
                }
            }
        }
    } else {
        tile_block_a<MA, MB, SG, ADJ, Acc, SrcE, MidE, OP, NC>(d, G, ip, sm, warp, nwarps, lane);
        if (!ip.black) __syncthreads();   // black is the same for the whole CTA
        tile_block_b<MA, MB, SG, ADJ, FIN, Acc, MidE, DstE, OP>(d, G, ip, sm, warp, nwarps, lane);
    }
}

}  // namespace fht
