// fht_batched.cuh -- the persistent batched-forward kernel: segment table
// layout, dependency counters and the item loop. Each (type, sign)
// instantiation lives in its own translation unit (batched_*.cu) so that
// they compile in parallel; fht_batched.cu holds the host-side plan.
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

struct BatchSeg {
    PassDesc d;          // lo/hi filled on the device from the image table / workspace
    int image, variant, m;
    int item_begin, tiles;
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

template <int MA, int MB, int SG, bool FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE>
__device__ __forceinline__ void run_item(const PassDesc &d, int gy, int tile, unsigned char *sm) {
    fused_forward_item<MA, MB, SG, false, FIN, Acc, SrcE, MidE, DstE>(
        d, gy, tile, reinterpret_cast<MidE *>(sm));
}

template <int SG, bool FIN, typename Acc, typename SrcE, typename MidE, typename DstE>
__device__ __forceinline__ void run_item_m(int m, const PassDesc &d, int gy, int tile,
                                           unsigned char *sm) {
    switch (m) {
    case 0: run_item<0, 0, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    case 1: run_item<1, 0, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    case 2: run_item<2, 0, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    case 3: run_item<3, 0, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    case 4: run_item<3, 1, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    case 5: run_item<3, 2, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    default: run_item<3, 3, SG, FIN, Acc, SrcE, MidE, DstE>(d, gy, tile, sm); break;
    }
}

// one batch = one quadrant, so one sign: the kernel is instantiated per sign
template <bool F32, int SG>
__global__ void __launch_bounds__(kWarps * 32, 2)
    batched_forward_kernel(const BatchSeg *segs, int n_segs, int total_items,
                           const fht_image_desc *descs, unsigned char *ws, Counters *ctr,
                           unsigned int *done, long long wait_budget, int dep_bias) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_seg, s_skip;
    __shared__ PassDesc s_desc;   // the current item's pass, pointers patched
    __shared__ int s_begin[kMaxSegsShared];   // segment start items, for the search
    const bool keys_shared = n_segs <= kMaxSegsShared;
    if (keys_shared)
        for (int i = threadIdx.x; i < n_segs; i += blockDim.x) s_begin[i] = segs[i].item_begin;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&ctr->next_item, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        if (threadIdx.x == 0) {
            // the segment holding this item (segments are sorted by item_begin)
            int lo = 0, hi = n_segs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                const int b = keys_shared ? s_begin[mid] : segs[mid].item_begin;
                if (b <= item) lo = mid;
                else hi = mid - 1;
            }
            s_seg = lo;
            int skip = 0;
            const BatchSeg &sg = segs[lo];
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
        __syncthreads();
        {
            // all threads copy the pass descriptor, then one patches its pointers
            const int *src = reinterpret_cast<const int *>(&segs[s_seg].d);
            int *dst = reinterpret_cast<int *>(&s_desc);
            for (int i = threadIdx.x; i < (int)(sizeof(PassDesc) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0 && !s_skip) {
            const BatchSeg &sg = segs[s_seg];
            const fht_image_desc &im = descs[sg.image];
            s_desc.lo.ptr = sg.lo_from_image ? const_cast<void *>(im.img) : (void *)(ws + sg.lo_off);
            if (sg.lo_from_image) s_desc.lo.pitch = im.img_pitch;
            s_desc.hi.ptr = sg.hi_from_image ? im.out : (void *)(ws + sg.hi_off);
            if (sg.hi_from_image) s_desc.hi.pitch = im.out_pitch;
        }
        __syncthreads();
        const BatchSeg &sg = segs[s_seg];
        if (!s_skip) {
            const PassDesc &d = s_desc;
            const int local = item - sg.item_begin;
            const int gy = local / sg.tiles, tile = local - gy * sg.tiles;
            if constexpr (F32) {
                if (d.hi_final)
                    run_item_m<SG, true, float, float, float, float>(sg.m, d, gy, tile, smem_raw);
                else
                    run_item_m<SG, false, float, float, float, float>(sg.m, d, gy, tile, smem_raw);
            } else {
                // a uint8 image is finished in one pass or goes to a uint16
                // level; a uint16 level's pass is the last (two passes at most)
                switch (sg.variant) {
                case kVarU8Final:
                    run_item_m<SG, true, int32_t, uint8_t, uint16_t, int32_t>(sg.m, d, gy, tile,
                                                                             smem_raw);
                    break;
                case kVarU8Level:
                    run_item_m<SG, false, int32_t, uint8_t, uint16_t, uint16_t>(sg.m, d, gy, tile,
                                                                               smem_raw);
                    break;
                default:
                    run_item_m<SG, true, int32_t, uint16_t, int32_t, int32_t>(sg.m, d, gy, tile,
                                                                             smem_raw);
                    break;
                }
            }
        }
        // make this item's stores visible GPU-wide before announcing it
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && !s_skip) atomicAdd(done + sg.done_index, 1u);
    }
}


using Kernel = void (*)(const BatchSeg *, int, int, const fht_image_desc *, unsigned char *,
                        Counters *, unsigned int *, long long, int);

// The four instantiations, one per translation unit.
Kernel kernel_f32_pos();
Kernel kernel_f32_neg();
Kernel kernel_u8_pos();
Kernel kernel_u8_neg();

}  // namespace batched
}  // namespace fht
