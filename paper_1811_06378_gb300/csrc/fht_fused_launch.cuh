// fht_fused_launch.cuh -- kernel wrapper and host launcher templates of the
// fused forward pass (included once per element-type translation unit).
#pragma once

#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "fht_fused.cuh"
#include "fht_host.h"
#include "fht_staged.cuh"

namespace fht {

#ifndef FHT_FUSED_WARPS
#define FHT_FUSED_WARPS 8
#endif
// Warps per CTA of the fused pass; CTAs per SM are sized to 16 warps.
constexpr int kFusedWarps = FHT_FUSED_WARPS;
// Largest dynamic shared memory one block may opt in to on sm_100-class parts.
constexpr size_t kMaxTileSmem = 227 * 1024;

// Bytes a pass must read and write at least: its source level as stored
// (image, or compact intermediate rows of the launched groups) and its
// destination (intermediate rows, output slopes, or image gradient).
// Launches of a range transform (PassDesc::range_call) are named with a
// "_range" suffix so that per-launch timings of range transforms and of
// whole quadrants can be told apart.
inline const char *range_suffix(const PassDesc &d) { return d.range_call ? "_range" : ""; }

inline double pass_alg_bytes(const PassDesc &d, int M, size_t src_bytes, size_t dst_bytes) {
    const double rows = (double)d.s_count * d.a_count * (1 << M);
    double rd, wr;
    if (d.lo_image) {
        rd = d.cyclic && !d.shear_on
                 ? (double)(d.src_t_last - d.src_t_first + 1) * d.W * src_bytes
                 : (double)d.lo.rows * d.lo.cols * src_bytes;
    } else {
        rd = rows * (d.lo_win ? d.win_len : d.lo.cols) * src_bytes;
    }
    if (!d.hi_final) {
        wr = rows * (d.hi_win ? d.win_len : d.hi.cols) * dst_bytes;
    } else if (d.dst_image) {
        wr = (double)(d.dst_h - d.dst_row_lo) * d.dst_w * dst_bytes * (d.accumulate ? 2 : 1);
    } else {
        const int t0 = d.a_lo << M, t1 = ((d.a_lo + d.a_count) << M) - 1;
        const int lo = t0 > d.t_first ? t0 : d.t_first, hi = t1 < d.t_last ? t1 : d.t_last;
        wr = hi >= lo ? (double)(hi - lo + 1) * d.W * dst_bytes : 0.0;
    }
    return rd + wr;
}

// SG is the pass's sign in buffer coordinates (+1 or -1) and FIN what it
// writes (0 an intermediate level, 1 the final level, 2 the final level of
// an adjoint into a transposed image gradient), both fixed at compile time.
// CTAs per SM the register budget is sized for: three (24 warps). A shared
// tile ends at the last column a stored lane reads (tile_geom), so a 2-byte
// tile (51 KB) or a 4-byte one of a 3 + 3-level pass (74 KB) fits three times.
// For 4-byte passes the 80 registers this leaves cost a few spills; measured
// at 4096^2, the final int32 pass still gains 2% over two CTAs at 120
// registers.
template <typename MidE>
constexpr int fused_min_blocks() {
    return 24 / kFusedWarps;
}

// The cyclic (adjoint-form) passes run at two CTAs per SM (128 registers):
// at 80 the final ones, whose image-gradient stores hold the old values of
// several rows, spill about 0.5 KB per thread, and the adjoint's first pass
// from an FP32 gradient ran 8% slower at three (4096^2: 62.7 -> 67.7 us). The
// first passes of the sheared and scaled transforms, from a uint8 image or a
// uint16 level into a level, gain at three (the +-15 degree sheared quadrant
// 84.0 -> 80.6 us).
template <int FIN, typename SrcE>
constexpr int adjoint_min_blocks() {
    return (FIN == 0 && sizeof(SrcE) < 4 ? 24 : 16) / kFusedWarps;
}

template <int MA, int MB, int SG, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE, int OP = 0>
__global__ void __launch_bounds__(kFusedWarps * 32, fused_min_blocks<MidE>())
    fused_forward_kernel(PassDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_forward_item<MA, MB, SG, false, FIN, Acc, SrcE, MidE, DstE, OP>(
        d, blockIdx.y, blockIdx.x, reinterpret_cast<MidE *>(smem_raw));
}

template <int MA, int MB, int SG, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE>
__global__ void __launch_bounds__(kFusedWarps * 32, adjoint_min_blocks<FIN, SrcE>())
    fused_adjoint_kernel(PassDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_forward_item<MA, MB, SG, true, FIN, Acc, SrcE, MidE, DstE>(
        d, blockIdx.y, blockIdx.x, reinterpret_cast<MidE *>(smem_raw));
}

// Uniform batch: image blockIdx.z of `d.batch` same-size transforms. The
// CTA's pass descriptor, with that image's source and destination, lives in
// shared memory (thread 0 writes it) and the item reads it there. (A local
// copy of the parameter with the two pointers changed goes to the stack.)
template <int MA, int MB, int SG, int FIN, bool ADJ, typename Acc, typename SrcE, typename MidE,
          typename DstE>
__global__ void __launch_bounds__(kFusedWarps * 32,
                                  ADJ ? adjoint_min_blocks<FIN, SrcE>() : fused_min_blocks<MidE>())
    fused_batch_kernel(PassDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ PassDesc s_d;
    if (threadIdx.x == 0) {
        s_d = d;
        s_d.lo.ptr = static_cast<char *>(d.lo.ptr) + (int64_t)blockIdx.z * d.lo_bstride;
        s_d.hi.ptr = static_cast<char *>(d.hi.ptr) + (int64_t)blockIdx.z * d.hi_bstride;
    }
    __syncthreads();
    fused_forward_item<MA, MB, SG, ADJ, FIN, Acc, SrcE, MidE, DstE>(
        s_d, blockIdx.y, blockIdx.x, reinterpret_cast<MidE *>(smem_raw));
}

template <int MA, int MB, bool ADJ, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE>
void (*batch_kernel_ptr(int sigma))(PassDesc) {
    return sigma > 0 ? fused_batch_kernel<MA, MB, 1, FIN, ADJ, Acc, SrcE, MidE, DstE>
                     : fused_batch_kernel<MA, MB, -1, FIN, ADJ, Acc, SrcE, MidE, DstE>;
}

// Uniform batches are built for float transforms (the differentiable path).
template <typename Acc, typename SrcE>
constexpr bool kBatchable = std::is_same<Acc, float>::value && std::is_same<SrcE, float>::value;

// Which final-level flags a type combination can take: uint16 is only ever an
// intermediate level, and a uint8 image goes to int32 only in a single
// (final) pass.
template <bool ADJ, typename SrcE, typename DstE>
struct FinCases {
    static constexpr bool kLevel = !(!ADJ && std::is_same<SrcE, uint8_t>::value &&
                                     std::is_same<DstE, int32_t>::value);
    static constexpr bool kFinal = !std::is_same<DstE, uint16_t>::value;
};

template <int MA, int MB, bool ADJ, int FIN, typename Acc, typename SrcE, typename MidE,
          typename DstE, int OP = 0>
void (*fused_kernel_ptr(int sigma))(PassDesc) {
    if constexpr (ADJ) {
        return sigma > 0 ? fused_adjoint_kernel<MA, MB, 1, FIN, Acc, SrcE, MidE, DstE>
                         : fused_adjoint_kernel<MA, MB, -1, FIN, Acc, SrcE, MidE, DstE>;
    } else {
        return sigma > 0 ? fused_forward_kernel<MA, MB, 1, FIN, Acc, SrcE, MidE, DstE, OP>
                         : fused_forward_kernel<MA, MB, -1, FIN, Acc, SrcE, MidE, DstE, OP>;
    }
}

// The staged persistent form of the final pass from a uint16 level
// (fht_staged.cuh): grid = SMs x resident CTAs, items taken in turn.
template <typename Dummy = void>
cudaError_t launch_staged(PassDesc d, cudaStream_t st) {
    set_debug_extents(d);
    const TileGeom G = tile_geom(3, 3, 1, 8, 1);
    const int tile_bytes = (1 << 6) * G.pitch * (int)sizeof(int32_t);
    const size_t smem = (size_t)tile_bytes + 8 * kStageWarpElems * sizeof(uint16_t);
    d.tile_w = G.tile_out;
    d.tiles = (d.p_count + G.tile_out - 1) / G.tile_out;
    const long long items = (long long)d.tiles * d.s_count * d.a_count;
    if (items == 0) return cudaSuccess;
    if (items > INT32_MAX) return cudaErrorInvalidValue;
    void (*k)(PassDesc, int, int) =
        d.sigma > 0 ? fused_staged_kernel<1> : fused_staged_kernel<-1>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 8 * 32, smem)) !=
        cudaSuccess)
        return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(items < slots ? items : slots);
    LaunchScope scope(d.range_call ? "forward_fused_m6_i32_final_range"
                                   : "forward_fused_m6_i32_final",
                      st, pass_alg_bytes(d, 6, 2, 4));
    k<<<grid, 8 * 32, smem, st>>>(d, (int)items, tile_bytes);
    scope.done();
    return cudaGetLastError();
}

template <int MA, int MB, bool ADJ, typename Acc, typename SrcE, typename MidE, typename DstE,
          int OP = 0>
cudaError_t launch_fused_t(PassDesc d, cudaStream_t st) {
    static_assert(OP == 0 || !ADJ, "max / min transforms have no adjoint");
    if (d.batch < 1 || d.batch > 65535) return cudaErrorInvalidValue;
    set_debug_extents(d);
    if constexpr (!kBatchable<Acc, SrcE> || OP != 0) {
        if (d.batch > 1) return cudaErrorNotSupported;
    }
    if constexpr (!ADJ && OP == 0 && MA == 3 && MB == 3 && std::is_same<Acc, int32_t>::value &&
                  std::is_same<SrcE, uint16_t>::value && std::is_same<MidE, int32_t>::value &&
                  std::is_same<DstE, int32_t>::value) {
        if (d.hi_final && !d.lo_image && d.batch == 1 && d.n_a == 1 && staged_enabled())
            return launch_staged(d, st);
    }
    TileGeom G = tile_geom(MA, MB, d.n_a, kFusedWarps, TilePad<MidE>::kPad);
    size_t smem = MB == 0 ? 0 : (size_t)(1 << (MA + MB)) * G.pitch * sizeof(MidE);
    // A tuned tile width that does not fit one block's shared memory is
    // narrowed until it does.
    while (smem > kMaxTileSmem && d.n_a > 1) {
        d.n_a--;
        G = tile_geom(MA, MB, d.n_a, kFusedWarps, TilePad<MidE>::kPad);
        smem = (size_t)(1 << (MA + MB)) * G.pitch * sizeof(MidE);
    }
    if (smem > kMaxTileSmem) return cudaErrorInvalidConfiguration;
    d.tile_w = G.tile_out;
    d.tiles = (d.p_count + G.tile_out - 1) / G.tile_out;
    dim3 grid(d.tiles, d.s_count * d.a_count, d.batch);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    using FC = FinCases<ADJ, SrcE, DstE>;
    void (*k)(PassDesc) = nullptr;
    const int fin = !d.hi_final ? 0 : (ADJ && d.dst_transpose ? 2 : 1);
    if (d.batch > 1) {
        if constexpr (kBatchable<Acc, SrcE> && OP == 0) {
            if (fin == 0) k = batch_kernel_ptr<MA, MB, ADJ, 0, Acc, SrcE, MidE, DstE>(d.sigma);
            else if (fin == 1) k = batch_kernel_ptr<MA, MB, ADJ, 1, Acc, SrcE, MidE, DstE>(d.sigma);
            else if constexpr (ADJ) k = batch_kernel_ptr<MA, MB, ADJ, 2, Acc, SrcE, MidE, DstE>(d.sigma);
        }
    } else if (d.hi_final) {
        if constexpr (FC::kFinal) {
            if constexpr (ADJ) {
                if (d.dst_transpose) k = fused_kernel_ptr<MA, MB, ADJ, 2, Acc, SrcE, MidE, DstE>(d.sigma);
            }
            if (!k) k = fused_kernel_ptr<MA, MB, ADJ, 1, Acc, SrcE, MidE, DstE, OP>(d.sigma);
        }
    } else {
        if constexpr (FC::kLevel)
            k = fused_kernel_ptr<MA, MB, ADJ, 0, Acc, SrcE, MidE, DstE, OP>(d.sigma);
    }
    if (!k) return cudaErrorInvalidValue;   // a type combination no plan produces
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    char name[64];
    snprintf(name, sizeof name, "%s_m%d_%s%s%s%s",
             d.shear_on ? "sheared_fused"
             : ADJ      ? "adjoint_fused"
             : OP == 1  ? "forward_max"
             : OP == 2  ? "forward_min"
                        : "forward_fused",
             MA + MB, acc_name<Acc>(), d.hi_final ? "_final" : "", d.batch > 1 ? "_batch" : "",
             range_suffix(d));
    LaunchScope scope(name, st,
                      d.batch * pass_alg_bytes(d, MA + MB, sizeof(SrcE), sizeof(DstE)));
    k<<<grid, kFusedWarps * 32, smem, st>>>(d);
    scope.done();
    return cudaGetLastError();
}

template <bool ADJ, typename Acc, typename SrcE, typename MidE, typename DstE, int OP = 0>
cudaError_t launch_fused_m(int M, const PassDesc &d, cudaStream_t st) {
    switch (M) {
    case 0: return launch_fused_t<0, 0, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    case 1: return launch_fused_t<1, 0, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    case 2: return launch_fused_t<2, 0, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    case 3: return launch_fused_t<3, 0, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    case 4: return launch_fused_t<3, 1, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    case 5: return launch_fused_t<3, 2, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    default: return launch_fused_t<3, 3, ADJ, Acc, SrcE, MidE, DstE, OP>(d, st);
    }
}

}  // namespace fht
