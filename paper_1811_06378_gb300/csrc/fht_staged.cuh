// fht_staged.cuh -- the final pass of a forward transform from a uint16 level
// (3 + 3 levels, int32 output) as a persistent kernel that stages block A's
// source rows in shared memory ahead of time.
//
// In the one-item-per-CTA pass, block A's eight warps wait on the L2 latency
// of their sheared source rows and then on each other at the CTA barrier.
// Here every warp owns a staging area for the 8 rows of its mini-strip; right
// after block A of item i has read them, the warp issues cp.async copies of
// item i+1's rows, which land while block B of item i runs. Block A then
// reads shared memory only. The item code (geometry, butterfly, block B,
// stores) is the same as the one-item-per-CTA kernel's, so the results are
// identical.
#pragma once

#include <cstdint>

#include "fht_fused.cuh"

namespace fht {

constexpr int kStageChunks = 34;                    // 16-byte chunks per staged row
constexpr int kStageRowElems = kStageChunks * 8;    // uint16 elements per staged row
constexpr int kStageWarpElems = 8 * kStageRowElems; // one warp's 8 rows

// 16-byte asynchronous copy global -> shared; the bytes past src_bytes are
// zero-filled (src_bytes = 0 reads nothing).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 :
                 : "r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Lowest level column the 32 lanes of a warp read from row s of group a
// (the 256 columns of one warp-column, sheared by a*s).
template <int SG>
__device__ __forceinline__ int staged_first_col(int A_off, int a, int s) {
    return SG > 0 ? A_off + a * s : A_off - a * s - (32 * kV - 1);
}

// Copy the 8 rows of mini-strip `warp` of item ip into the warp's staging
// area: per row, the 16-byte chunks from the 8-aligned column at or below the
// first one read, zero outside [0, lo.cols) (a chunk starts on a multiple of
// 8, so it is either wholly left of column 0 or starts inside the row).
template <int SG>
__device__ __forceinline__ void stage_rows(const PassDesc &d, const ItemPos &ip, int warp,
                                           int lane, uint16_t *stage) {
    constexpr int M = 6;
    const uint16_t *base = reinterpret_cast<const uint16_t *>(d.lo.ptr);
    for (int j = lane; j < 8 * kStageChunks; j += 32) {
        const int rho = j / kStageChunks, k = j - rho * kStageChunks;
        const int s = warp * 8 + rho;
        const int64_t row = ((((int64_t)ip.S << M) + s) << d.k0) + ip.a;
        const int c = (staged_first_col<SG>(ip.A_off, ip.a, s) & ~7) + 8 * k;
        int bytes = 0;
        if (c >= 0 && c < d.lo.cols) bytes = d.lo.cols - c >= 8 ? 16 : 2 * (d.lo.cols - c);
        const uint16_t *src = base + row * d.lo.pitch + (bytes > 0 ? c : 0);
        if (bytes > 0 && !FHT_LOAD_OK(src, bytes)) bytes = 0;
        cp_async16(stage + rho * kStageRowElems + 8 * k, src, bytes);
    }
    cp_async_commit();
}

// v[k] = staged row element off + k (uint16, 16-byte aligned row; off + 8
// lies inside the row): the two aligned chunks around it, realigned in
// registers as load8_fast does for global rows.
template <typename Acc>
__device__ __forceinline__ void load8_staged(const uint16_t *row, int off, Acc (&v)[kV]) {
    const int delta = off & 7;
    const uint4 *g = reinterpret_cast<const uint4 *>(row + (off & ~7));
    const uint4 q0 = g[0], q1 = g[1];
    const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
    const int jw = delta >> 1;
    uint32_t u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
        u[i] = sel4(w[i], w[i + 1 < 8 ? i + 1 : 7], w[i + 2 < 8 ? i + 2 : 7],
                    w[i + 3 < 8 ? i + 3 : 7], jw);
    const uint32_t sel = (delta & 1) ? 0x5432u : 0x3210u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t pr = __byte_perm(u[i], u[i + 1], sel);
        v[2 * i] = (Acc)(int32_t)(pr & 0xffffu);
        v[2 * i + 1] = (Acc)(int32_t)(pr >> 16);
    }
}

// Persistent final pass: item = blockIdx.x, blockIdx.x + gridDim.x, ...
// Shared memory: the tile, then 8 staging areas (one per warp).
template <int SG>
__global__ void __launch_bounds__(8 * 32, 2)
    fused_staged_kernel(PassDesc d, int n_items, int tile_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int MA = 3, MB = 3, M = MA + MB, RA = 1 << MA, PAD = 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TileGeom G = tile_geom(MA, MB, 1, 8, PAD);
    const int T = G.tile_out, P = G.pitch;
    int32_t *tile = reinterpret_cast<int32_t *>(smem_raw);
    uint16_t *stage = reinterpret_cast<uint16_t *>(smem_raw + tile_bytes) + warp * kStageWarpElems;
    const int tiles = d.tiles;
    FHT_DEBUG_BEGIN(d);
    int item = blockIdx.x;
    ItemPos ip{};
    if (item < n_items) {
        ip = item_pos<M, SG, false, 1>(d, T, item / tiles, item % tiles);
        if (!ip.black) stage_rows<SG>(d, ip, warp, lane, stage);
    }
    const int i0 = lane * kV;
    for (; item < n_items; item += gridDim.x) {
        const ItemPos cur = ip;
        if (!cur.black) {
            cp_async_wait_all();
            __syncwarp();
            int32_t v[RA][kV];
#pragma unroll
            for (int rho = 0; rho < RA; ++rho) {
                const int s = warp * RA + rho;
                const int cs = staged_first_col<SG>(cur.A_off, cur.a, s) & ~7;
                const int lo = SG > 0 ? cur.A_off + i0 + cur.a * s
                                      : cur.A_off - i0 - cur.a * s - (kV - 1);
                load8_staged<int32_t>(stage + rho * kStageRowElems, lo - cs, v[rho]);
                if constexpr (SG < 0) reverse8(v[rho]);
            }
            reg_butterfly<MA, int32_t>(v);
            if (lane < kLanesValid) {
                const int pos = (8 + PAD) * (i0 >> 3);
#pragma unroll
                for (int c = 0; c < RA; ++c) {
                    int32_t *row = tile + (warp * RA + c) * P + pos;
#pragma unroll
                    for (int k = 0; k < kV; ++k) row[k] = v[c][k];
                }
            }
        }
        __syncwarp();   // every lane has read the stage before it is refilled
        const int next = item + gridDim.x;
        if (next < n_items) {
            ip = item_pos<M, SG, false, 1>(d, T, next / tiles, next % tiles);
            if (!ip.black) stage_rows<SG>(d, ip, warp, lane, stage);
        }
        if (!cur.black) __syncthreads();   // the tile is complete (black is CTA-uniform)
        tile_block_b<MA, MB, SG, false, 1, int32_t, int32_t, int32_t>(d, G, cur, tile, warp, 8,
                                                                     lane);
        __syncthreads();   // block B has read the tile before the next block A writes it
    }
    cp_async_wait_all();
}

}  // namespace fht
