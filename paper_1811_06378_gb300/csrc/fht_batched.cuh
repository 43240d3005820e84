// fht_batched.cuh -- the persistent batched kernel (forward transforms and
// FP32 adjoints of many images of different sizes): segment table layout,
// dependency counters and the item loop. Each (mode, sign) instantiation
// lives in its own translation unit (batched_*.cu) so that they compile in
// parallel; fht_batched.cu holds the host-side plan.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fht.h"
#include "fht_fused.cuh"

namespace fht {
namespace batched {

constexpr int kWarps = 8;
constexpr int kMaxBatchK = 12;   // images up to 4096 rows (transposed: columns)
constexpr int kMaxSegsShared = 2048;   // segment keys kept in shared memory

// Kernel variants. uint8 -> int32: single-pass images, first passes into a
// uint16 level, and int32 final passes from it. float: one variant per M.
enum : int { kVarU8Final = 0, kVarU8Level = 10, kVarU16Final = 20, kVarF32 = 30 };

// What one launch runs: uint8 -> int32 forward transforms, float forward
// transforms, or float adjoints whose final level goes to the image gradient
// as is (quadrants Q0, Q1) or transposed (Q2, Q3).
enum : int { kModeU8 = 0, kModeF32 = 1, kModeAdj = 2, kModeAdjT = 3 };

struct BatchSeg {
    PassDesc d;          // complete; lo/hi pointers and pitches written by the host per call
    int image, variant, m;
    int item_begin, tiles;
    int units;           // (group, tile) units of the segment: s_count * a_count * tiles
    int chunk;           // consecutive units one item covers
    int done_index;      // counter of this (image, pass)
    int dep_index;       // counter of (image, pass - 1), or -1
    int dep_count;       // items of (image, pass - 1)
    int lo_from_image;   // lo is the caller's image, else workspace + lo_off
    int hi_from_image;   // hi is the caller's output, else workspace + hi_off
    int64_t lo_off, hi_off;
};

struct Counters {
    unsigned int next_item;
    int error;           // FHT_OK or FHT_ETIMEOUT
    unsigned int pad[2];
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// A pass that reads a level reads it with coherent loads (NC = false): its
// image's earlier pass wrote it in this same launch. Passes from the caller's
// image (NC = true) read it through the non-coherent path: nothing writes it.
template <int MA, int MB, int SG, bool ADJ, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE, bool NC>
__device__ __forceinline__ void run_item(const PassDesc &d, int gy, int tile, unsigned char *sm) {
    fused_forward_item<MA, MB, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, 0, NC>(
        d, gy, tile, reinterpret_cast<MidE *>(sm));
}

template <int SG, int FIN, typename Acc, typename SrcE, typename MidE, typename DstE,
          bool ADJ = false, bool NC = false>
__device__ __forceinline__ void run_item_m(int m, const PassDesc &d, int gy, int tile,
                                           unsigned char *sm) {
    switch (m) {
    case 0: run_item<0, 0, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    case 1: run_item<1, 0, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    case 2: run_item<2, 0, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    case 3: run_item<3, 0, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    case 4: run_item<3, 1, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    case 5: run_item<3, 2, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    default: run_item<3, 3, SG, ADJ, FIN, Acc, SrcE, MidE, DstE, NC>(d, gy, tile, sm); break;
    }
}

// one batch = one quadrant, so one sign: the kernel is instantiated per mode
// and sign (an adjoint's sign is the opposite of its quadrant's).
// Thread 0 claims the next item while the CTA works on the current one (the
// claim's latency is hidden), finds its segment and waits for its dependency;
// all threads then copy the segment's pass descriptor (complete, pointers
// included, written by the host) into shared memory. After an item one thread
// of the last warp alone fences and counts it done: the CTA barrier before it
// orders every thread's stores before that release.
// Holding one claimed item ahead keeps the waits finite: the smallest
// unfinished item is always some CTA's current item, and everything it
// depends on has a smaller index.
// MINB: CTAs per SM the register budget is sized for (2 or 3).
template <int MODE, int SG, int MINB>
__global__ void __launch_bounds__(kWarps * 32, MINB)
    batched_kernel(const BatchSeg *segs, int n_segs, int total_items, Counters *ctr,
                   unsigned int *done, long long wait_budget, int dep_bias) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_skip, s_m, s_variant, s_tiles, s_first, s_done, s_units, s_chunk;
    __shared__ int s_seg;
    __shared__ PassDesc s_desc;   // the current item's pass
    __shared__ int s_begin[kMaxSegsShared];   // segment start items, for the search
    const bool keys_shared = n_segs <= kMaxSegsShared;
    if (keys_shared)
        for (int i = threadIdx.x; i < n_segs; i += blockDim.x) s_begin[i] = segs[i].item_begin;
    int next = 0;   // thread 0: the claimed next item
    if (threadIdx.x == 0) next = (int)atomicAdd(&ctr->next_item, 1u);
    __syncthreads();   // s_begin complete
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = next;
            s_item = item;
            if (item < total_items) {
                next = (int)atomicAdd(&ctr->next_item, 1u);
                // the segment holding this item (segments are sorted by item_begin)
                int lo = 0, hi = n_segs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    const int b = keys_shared ? s_begin[mid] : segs[mid].item_begin;
                    if (b <= item) lo = mid;
                    else hi = mid - 1;
                }
                const BatchSeg &sg = segs[lo];
                s_seg = lo;
                s_m = sg.m;
                s_variant = sg.variant;
                s_tiles = sg.tiles;
                s_first = sg.item_begin;
                s_done = sg.done_index;
                s_units = sg.units;
                s_chunk = sg.chunk;
                int skip = 0;
                if (sg.dep_index >= 0) {
                    const unsigned int need = (unsigned int)(sg.dep_count + dep_bias);
                    const long long t0 = clock64();
                    while (ld_acquire(done + sg.dep_index) < need) {
                        __nanosleep(256);
                        if (clock64() - t0 > wait_budget) {
                            atomicExch(&ctr->error, (int)FHT_ETIMEOUT);
                            skip = 1;
                            break;
                        }
                    }
                }
                s_skip = skip;
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        {
            const int *src = reinterpret_cast<const int *>(&segs[s_seg].d);
            int *dst = reinterpret_cast<int *>(&s_desc);
            for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        const bool skip = s_skip != 0;
        const int done_at = s_done;   // thread 0 rewrites s_done for the next item
        if (!skip) {
            const PassDesc &d = s_desc;
            const int m = s_m, tiles = s_tiles;
            const int u0 = (item - s_first) * s_chunk;
            const int u1 = u0 + s_chunk < s_units ? u0 + s_chunk : s_units;
            for (int u = u0; u < u1; ++u) {
                if (u > u0) __syncthreads();   // the previous unit's reads of the shared tile
                const int gy = u / tiles, tile = u - gy * tiles;
                if constexpr (MODE == kModeAdj || MODE == kModeAdjT) {
                    // float adjoint: cyclic intermediate levels, image gradient last
                    if (d.hi_final)
                        run_item_m<SG, MODE == kModeAdjT ? 2 : 1, float, float, float, float,
                                   true>(m, d, gy, tile, smem_raw);
                    else
                        run_item_m<SG, 0, float, float, float, float, true>(m, d, gy, tile,
                                                                            smem_raw);
                } else if constexpr (MODE == kModeF32) {
                    if (d.hi_final)
                        run_item_m<SG, 1, float, float, float, float>(m, d, gy, tile, smem_raw);
                    else
                        run_item_m<SG, 0, float, float, float, float>(m, d, gy, tile, smem_raw);
                } else {
                    // a uint8 image is finished in one pass or goes to a uint16
                    // level; a uint16 level's pass is the last (two passes at most)
                    switch (s_variant) {
                    case kVarU8Final:
                        run_item_m<SG, 1, int32_t, uint8_t, uint16_t, int32_t, false, true>(
                            m, d, gy, tile, smem_raw);
                        break;
                    case kVarU8Level:
                        run_item_m<SG, 0, int32_t, uint8_t, uint16_t, uint16_t, false, true>(
                            m, d, gy, tile, smem_raw);
                        break;
                    default:
                        run_item_m<SG, 1, int32_t, uint16_t, int32_t, int32_t>(m, d, gy, tile,
                                                                              smem_raw);
                        break;
                    }
                }
            }
        }
        __syncthreads();   // every thread's stores of this item precede the release below
        // The release is made by the last warp, so that its fence overlaps
        // thread 0's claim, search and wait for the next item.
        if (threadIdx.x == (kWarps - 1) * 32 && !skip) {
            __threadfence();
            atomicAdd(done + done_at, 1u);
        }
    }
}

using Kernel = void (*)(const BatchSeg *, int, int, Counters *, unsigned int *, long long, int);

// The instantiations, one per translation unit: forward transforms per type
// and sign; adjoints per quadrant (sign, and whether the image gradient is
// transposed); each for 2 or 3 CTAs per SM (minb).
Kernel kernel_f32_pos(int minb);
Kernel kernel_f32_neg(int minb);
Kernel kernel_u8_pos(int minb);
Kernel kernel_u8_neg(int minb);
Kernel kernel_adj_q0(int minb);
Kernel kernel_adj_q1(int minb);
Kernel kernel_adj_q2(int minb);
Kernel kernel_adj_q3(int minb);

}  // namespace batched
}  // namespace fht
