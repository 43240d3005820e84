// fht_host.h -- host-side declarations shared by the library's translation
// units: launch accounting and the per-type fused-pass launchers.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "fht_common.cuh"

namespace fht {

// Counts a kernel launch and, while profiling is on (fht_profile_begin),
// brackets it with CUDA events on its stream: construct right before the
// launch, call done() right after it. With FHT_NVTX=1 in the environment when
// the library loads, every launch is also an NVTX range named after the
// kernel (for nsys / ncu --nvtx filtering); off by default. alg_bytes: the bytes the launch must
// move at least (the level it reads as stored plus the level it writes).
class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t st, double alg_bytes);
    void done();

  private:
    cudaStream_t st_;
    double bytes_;
    bool on_ = false;
    bool nvtx_ = false;   // an NVTX range was pushed for this launch (FHT_NVTX=1)
    std::string name_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Device-side error counters (one per translation unit that holds kernels
// able to record one): each registers a function that returns its count and
// resets it; read_device_counters sums them. Registration returns true so it
// can initialise a namespace-scope constant.
bool register_device_counter(unsigned int (*read_and_reset)());
unsigned int read_device_counters();

// Whether the final pass from a uint16 level runs as the staged persistent
// kernel (fht_staged.cuh; FHT_STAGED=0 in the environment turns it off).
bool staged_enabled();

// Bytes the debug build's test hook takes off every destination span
// (fht_debug_test_hooks; 0 normally).
long long debug_hi_shrink();

inline size_t elem_size(int type) { return type == kU8 ? 1 : type == kU16 ? 2 : 4; }

// The spans a pass may touch (PassDesc::dbg_lo_bytes / dbg_hi_bytes), from
// the descriptor's own geometry: a level buffer is n rows of its pitch; the
// caller's image is its rows x columns view (transposed for Q2/Q3); a
// gradient source covers the rows its row map reaches; a destination covers
// the rows and columns its map writes. Only the debug build reads them.
inline void set_debug_extents(PassDesc &d) {
    const long long le = (long long)elem_size(d.lo.type), he = (long long)elem_size(d.hi.type);
    long long lo = 0, hi = 0;
    if (!d.lo_image) {
        lo = (long long)d.n * d.lo.pitch * le;
    } else if (d.cyclic && !d.shear_on) {
        const long long r0 = d.src_row_base + (long long)d.src_row_dir * d.src_t_first;
        const long long r1 = d.src_row_base + (long long)d.src_row_dir * d.src_t_last;
        lo = ((r0 > r1 ? r0 : r1) * d.lo.pitch + d.W) * le;
    } else {
        const long long cols = d.lo.cols;
        const long long mr = d.transpose ? cols : d.lo.rows, mc = d.transpose ? d.lo.rows : cols;
        lo = ((mr - 1) * d.lo.pitch + mc) * le;
    }
    if (!d.hi_final) {
        hi = (long long)d.n * d.hi.pitch * he;
    } else if (d.dst_image) {
        const long long rows = d.dst_transpose ? d.dst_w : d.dst_h - d.dst_row_lo;
        const long long cols = d.dst_transpose ? d.dst_h : d.dst_w;
        hi = ((rows - 1) * d.hi.pitch + cols) * he;
    } else {
        const long long r0 = d.row_base + (long long)d.row_dir * d.t_first;
        const long long r1 = d.row_base + (long long)d.row_dir * d.t_last;
        hi = ((r0 > r1 ? r0 : r1) * d.hi.pitch + d.W) * he;
    }
    d.dbg_lo_bytes = lo > 0 ? lo : 0;
    hi -= debug_hi_shrink();
    d.dbg_hi_bytes = hi > 0 ? hi : 0;
}

// Window of the level an adjoint's final pass reads (final pass of Mf levels,
// cropped to the w_c columns p in [p_begin, p_begin + w_c), p_begin = n for
// sign +1 and 0 for sign -1): row (s, a) is read on the w_c + 2^Mf - 1
// columns from c + sigma*a*s, c = 2^(K - Mf) for sign +1 (the final level's
// columns sit 2^K - 2^(K - Mf) past the level's) and -(2^Mf - 1) for sign -1.
// The stored window starts 8 to 15 columns earlier (win_base), so it is 15
// columns longer, rounded up to 8. 0 when the window would not save anything
// (it must stay 16 columns short of W).
inline void adjoint_window(int w_c, int W, int K, int Mf, int sigma, int *len, int *c) {
    const int L = (w_c + (1 << Mf) - 1 + 15 + 7) / 8 * 8;
    *len = 0;
    *c = 0;
    if (L + 16 > W) return;
    *len = L;
    *c = sigma > 0 ? (1 << (K - Mf)) : W - ((1 << Mf) - 1);
}

template <typename T> inline const char *acc_name();
template <> inline const char *acc_name<float>() { return "f32"; }
template <> inline const char *acc_name<int32_t>() { return "i32"; }

// Fused forward pass of M levels, one launcher per (accumulator, source,
// destination) element-type combination; each lives in its own translation
// unit so the instantiations compile in parallel.
cudaError_t launch_fused_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_fused_i32_u8_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_fused_i32_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_fused_i32_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_fused_f32_u8(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_fused_f32_f32(int M, const PassDesc &d, cudaStream_t st);
// Adjoint passes: the opposite-sign cyclic transform of a gradient.
cudaError_t launch_adjoint_f32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_adjoint_i32(int M, const PassDesc &d, cudaStream_t st);
// The same cyclic pass code over a uint8 image: first passes of the sheared
// forward transform.
cudaError_t launch_adjoint_f32_u8(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_adjoint_i32_u8(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_adjoint_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_adjoint_i32_u16(int M, const PassDesc &d, cudaStream_t st);
// Forward passes with the maximum / minimum along the patterns (OP 1 / 2).
cudaError_t launch_max_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_max_i32_u8_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_max_i32_u16_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_max_i32_u16_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_max_f32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_min_i32_u8_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_min_i32_u8_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_min_i32_u16_u16(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_min_i32_u16_i32(int M, const PassDesc &d, cudaStream_t st);
cudaError_t launch_min_f32(int M, const PassDesc &d, cudaStream_t st);

// Nearest-neighbour scale of a rows x cols image (elements of elem bytes,
// pitches in elements) by the 32.32 step D along one axis (Section 4):
// dst[r][c] = src[r][(c * D) >> 32] (along_rows false: every row scaled to
// out_cols columns) or src[(r * D) >> 32][c] (true: out_rows rows, each a
// copy of its source row). Every source index stays below the source's
// extent when out_cols (out_rows) is the scaled width of fht_scaled_width.
cudaError_t launch_scale_image(const void *src, int64_t src_pitch, int elem, bool along_rows,
                               long long D, void *dst, int64_t dst_pitch, int out_rows,
                               int out_cols, cudaStream_t st);

}  // namespace fht
