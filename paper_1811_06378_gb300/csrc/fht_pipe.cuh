// fht_pipe.cuh -- the two-block pass as a persistent, warp-specialised
// pipeline.
//
// A CTA of two groups of kPipeGroupWarps warps loops over its items
// (blockIdx.x, + gridDim.x, ...). The producer group runs block A of each item
// (global loads, MA levels, shared tile); the consumer group runs block B
// (sheared tile reads, MB levels, destination stores). Two shared tiles
// alternate between items, so while the consumers work on item k the
// producers already load item k+1: the global-load latency of block A is
// covered by block B's work instead of stalling every warp at a CTA barrier.
//
// Hand-off per tile buffer b uses two mbarriers, each completed by the
// arrivals of all threads of one group:
//   full[b]  -- producers finished writing the tile (consumers wait on it);
//   empty[b] -- consumers finished reading it (producers wait before reuse).
// The j-th use of buffer b waits for phase parity j & 1 of full[b], and (for
// j >= 1) for parity (j - 1) & 1 of empty[b]; a group is never more than one
// use of a buffer ahead of the other, so no phase is lapped. Every wait is
// bounded by a clock budget: past it the thread counts a timeout in a device
// counter and leaves, so a launch always ends.
#pragma once

#include "fht_fused.cuh"

namespace fht {

constexpr int kPipeGroupWarps = 8;
constexpr int kPipeThreads = 2 * kPipeGroupWarps * 32;
constexpr long long kPipeWaitBudget = 2000000000LL;   // SM clocks, about a second

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// arrive with release semantics at CTA scope (orders this thread's tile writes
// or reads before the phase completes)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete; false once the clock
// budget is spent.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kPipeWaitBudget) return false;
    return true;
}

// Bytes of one shared tile, rounded to 128 (the second tile keeps the first's alignment).
__host__ __device__ inline size_t pipe_tile_bytes(const TileGeom &G, int MA, int MB,
                                                  size_t mid_bytes) {
    const size_t b = (size_t)(1 << (MA + MB)) * G.pitch * mid_bytes;
    return (b + 127) & ~(size_t)127;
}

template <int MA, int MB, int SG, bool ADJ, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE>
__device__ __forceinline__ void pipe_items(const PassDesc &d, int n_items, size_t tile_bytes,
                                           unsigned char *smem, uint64_t *bars,
                                           unsigned int *timeouts) {
    constexpr int M = MA + MB;
    constexpr int PAD = TilePad<MidE>::kPad;
    constexpr unsigned kGroupThreads = kPipeGroupWarps * 32;
    const TileGeom G = tile_geom(MA, MB, d.n_a, kPipeGroupWarps, PAD);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(&bars[b], kGroupThreads);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp < kPipeGroupWarps;
    const int gw = producer ? warp : warp - kPipeGroupWarps;
    int k = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
        const int b = k & 1;
        const unsigned use = (unsigned)k >> 1;   // earlier uses of buffer b
        MidE *sm = reinterpret_cast<MidE *>(smem + b * tile_bytes);
        const int gy = item / d.tiles, tile = item - gy * d.tiles;
        const ItemPos ip = item_pos<M, SG, ADJ, FIN>(d, G.tile_out, gy, tile);
        if (producer) {
            if (use > 0 && !mbar_wait(&bars[2 + b], (use - 1) & 1u)) {
                atomicAdd(timeouts, 1u);
                return;
            }
            tile_block_a<MA, MB, SG, ADJ, Acc, SrcE, MidE>(d, G, ip, sm, gw, kPipeGroupWarps,
                                                           lane);
            mbar_arrive(&bars[b]);
        } else {
            if (!mbar_wait(&bars[b], use & 1u)) {
                atomicAdd(timeouts, 1u);
                return;
            }
            tile_block_b<MA, MB, SG, ADJ, FIN, Acc, MidE, DstE>(d, G, ip, sm, gw,
                                                                kPipeGroupWarps, lane);
            mbar_arrive(&bars[2 + b]);
        }
    }
}

}  // namespace fht
