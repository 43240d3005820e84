// fht_api.cu -- C ABI (include/fht.h): argument checks, pass planning and
// kernel launches for the GB300 fast Hough transform.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fht.h"
#include "fht_kernels.cuh"

using namespace fht;

namespace {

thread_local int g_last_cuda_error = 0;

// ------------------------------------------------------------ launch profiling
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Counts a launch and, while profiling is on, brackets it with events on its
// stream: construct right before the launch, call done() right after.
class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t st) : st_(st) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        on_ = g_prof_on;
        if (on_) {
            rec_.name = name;
            rec_.a = take_event();
            rec_.b = take_event();
            cudaEventRecord(rec_.a, st_);
        }
    }
    void done() {
        if (!on_) return;
        cudaEventRecord(rec_.b, st_);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back(rec_);
        on_ = false;
    }

  private:
    cudaStream_t st_;
    bool on_ = false;
    ProfRec rec_;
};

template <typename T> const char *acc_name();
template <> const char *acc_name<float>() { return "f32"; }
template <> const char *acc_name<int32_t>() { return "i32"; }

constexpr int kBlock = 256;
constexpr int kMaxLevelsPerPass = 6;
constexpr int kMaxK = 15;            // n <= 32768
constexpr int kMaxSide = 32768;

int next_pow2(int v) {
    int n = 1;
    while (n < v) n *= 2;
    return n;
}
int ilog2(int n) {
    int k = 0;
    while ((1 << k) < n) ++k;
    return k;
}
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Acc type of a (input, accumulator) pair; -1 if unsupported.
int acc_kind(fht_dtype in_t, fht_dtype acc_t) {
    if (acc_t == FHT_I32 && (in_t == FHT_U8 || in_t == FHT_I32)) return kI32;
    if (acc_t == FHT_F32 && (in_t == FHT_U8 || in_t == FHT_F32)) return kF32;
    return -1;
}
int elem_of(fht_dtype t) { return t == FHT_U8 ? kU8 : t == FHT_I32 ? kI32 : kF32; }
size_t elem_bytes(int e) { return e == kU8 ? 1 : e == kU16 ? 2 : 4; }

// Split K levels into passes of at most kMaxLevelsPerPass, as even as possible,
// larger passes first.
int split_levels(int K, int *m) {
    if (K == 0) { m[0] = 0; return 1; }
    int P = (K + kMaxLevelsPerPass - 1) / kMaxLevelsPerPass;
    for (int p = 0; p < P; ++p) m[p] = K / P + (p < K % P ? 1 : 0);
    return P;
}

// Geometry and pass plan of one quadrant transform.
struct QuadPlan {
    int q, sigma, transpose;
    int h_c, w_c;       // content size of the (transposed) image
    int n, K, W;
    int w_in;           // meaningful width used by fhtshift
    int npass;
    int m[4], k[5];
    int lvl_type[5];    // element type of intermediate level k[p] (1 <= p < npass)
    int lvl_cols[5];
    int64_t lvl_pitch[5];
    size_t buf_bytes[2];
};

QuadPlan make_plan(int h, int w, int q, bool full, int in_elem, int acc_elem) {
    QuadPlan P{};
    P.q = q;
    P.transpose = q >= 2;
    P.sigma = (q == 0 || q == 3) ? 1 : -1;
    P.h_c = P.transpose ? w : h;
    P.w_c = P.transpose ? h : w;
    P.n = next_pow2(P.h_c);
    P.K = ilog2(P.n);
    if (full) {
        P.W = next_pow2(h) + next_pow2(w);
        P.w_in = P.W - P.n;
    } else {
        P.W = P.w_c + P.n;
        P.w_in = P.w_c;
    }
    P.npass = split_levels(P.K, P.m);
    P.k[0] = 0;
    for (int p = 0; p < P.npass; ++p) P.k[p + 1] = P.k[p] + P.m[p];
    P.buf_bytes[0] = P.buf_bytes[1] = 0;
    for (int p = 1; p < P.npass; ++p) {
        int k = P.k[p];
        int type = acc_elem;
        // u8 images summed over 2^k rows stay below 2^16 while k <= 8
        if (acc_elem == kI32 && in_elem == kU8 && k <= 8) type = kU16;
        P.lvl_type[p] = type;
        P.lvl_cols[p] = std::min(P.W, P.w_c + (1 << k));
        P.lvl_pitch[p] = (int64_t)align_up(P.lvl_cols[p], 64);
        size_t bytes = align_up((size_t)P.n * P.lvl_pitch[p] * elem_bytes(type), 256);
        size_t &slot = P.buf_bytes[(p - 1) % 2];
        slot = std::max(slot, bytes);
    }
    return P;
}

size_t plan_workspace(const QuadPlan &P) { return P.buf_bytes[0] + P.buf_bytes[1]; }

void *level_ptr(const QuadPlan &P, void *ws, int p) {
    char *base = (char *)ws;
    return (p - 1) % 2 == 0 ? base : base + P.buf_bytes[0];
}

// Where the final level goes.
struct FinalMap {
    int t_first, t_last, row_base, row_dir;
    int shift_on, shift_inverse;
};

// Quadrant layout: slope t is output row t - t_lo (t_lo = 0 unless a range).
FinalMap quadrant_map(int t_lo, int t_hi) { return FinalMap{t_lo, t_hi, -t_lo, 1, 0, 0}; }

// Full layout (Section 3.3): Q0 flipped rows [0, hp), Q1 t >= 1 next, Q2
// flipped without its 45-degree row, Q3 t >= 1 last.
FinalMap full_map(int q, int hp, int wp) {
    switch (q) {
    case 0: return FinalMap{0, hp - 1, hp - 1, -1, 0, 0};
    case 1: return FinalMap{1, hp - 1, hp - 1, 1, 0, 0};
    case 2: return FinalMap{0, wp - 2, 2 * hp + wp - 3, -1, 0, 0};
    default: return FinalMap{1, wp - 1, 2 * hp + wp - 3, 1, 0, 0};
    }
}

int tile_width(int M) { return M >= 4 ? 128 : 256; }

template <int M, typename AccT>
__global__ void __launch_bounds__(kBlock) forward_pass_kernel(PassDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    forward_item<M, AccT>(d, blockIdx.y, blockIdx.x, reinterpret_cast<AccT *>(smem_raw));
}

template <int M, typename AccT>
__global__ void __launch_bounds__(kBlock) adjoint_pass_kernel(PassDesc d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    adjoint_item<M, AccT>(d, blockIdx.y, blockIdx.x, reinterpret_cast<AccT *>(smem_raw));
}

template <int M, typename AccT>
cudaError_t launch_pass_t(const PassDesc &d, bool adjoint, cudaStream_t st) {
    size_t smem = (size_t)item_smem_elems(M, d.tile_w) * sizeof(AccT);
    dim3 grid(d.tiles, d.s_count * d.a_count);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    char name[64];
    snprintf(name, sizeof name, "%s_pass_m%d_%s%s", adjoint ? "adjoint" : "forward", M,
             acc_name<AccT>(),
             adjoint ? (d.lo_image ? "_to_image" : "") : (d.hi_final ? "_final" : ""));
    auto k = adjoint ? adjoint_pass_kernel<M, AccT> : forward_pass_kernel<M, AccT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    LaunchScope scope(name, st);
    k<<<grid, kBlock, smem, st>>>(d);
    scope.done();
    return cudaGetLastError();
}

template <typename AccT>
cudaError_t launch_pass(int M, const PassDesc &d, bool adjoint, cudaStream_t st) {
    switch (M) {
    case 0: return launch_pass_t<0, AccT>(d, adjoint, st);
    case 1: return launch_pass_t<1, AccT>(d, adjoint, st);
    case 2: return launch_pass_t<2, AccT>(d, adjoint, st);
    case 3: return launch_pass_t<3, AccT>(d, adjoint, st);
    case 4: return launch_pass_t<4, AccT>(d, adjoint, st);
    case 5: return launch_pass_t<5, AccT>(d, adjoint, st);
    default: return launch_pass_t<6, AccT>(d, adjoint, st);
    }
}

// Fill the pass descriptor shared by forward and adjoint: pass p of plan P.
PassDesc pass_desc(const QuadPlan &P, int p, const Side &image, const Side &final_side,
                   void *ws, const FinalMap &fm, int t_lo, int t_hi) {
    PassDesc d{};
    d.lo_image = p == 0;
    d.transpose = P.transpose;
    if (p == 0) {
        d.lo = image;
    } else {
        d.lo = Side{level_ptr(P, ws, p), P.lvl_pitch[p], P.lvl_type[p], P.n, P.lvl_cols[p]};
    }
    d.hi_final = p == P.npass - 1;
    if (d.hi_final) {
        d.hi = final_side;
        d.hi.cols = P.W;
    } else {
        d.hi = Side{level_ptr(P, ws, p + 1), P.lvl_pitch[p + 1], P.lvl_type[p + 1], P.n,
                    P.lvl_cols[p + 1]};
    }
    d.n = P.n;
    d.W = P.W;
    d.K = P.K;
    d.k0 = P.k[p];
    d.sigma = P.sigma;
    int drop = P.K - P.k[p];
    d.a_lo = t_lo >> drop;
    d.a_count = (t_hi >> drop) - d.a_lo + 1;
    d.s_count = P.n >> P.k[p + 1];
    d.tile_w = tile_width(P.m[p]);
    d.tiles = (d.hi.cols + d.tile_w - 1) / d.tile_w;
    d.t_first = fm.t_first;
    d.t_last = fm.t_last;
    d.row_base = fm.row_base;
    d.row_dir = fm.row_dir;
    d.shift_on = fm.shift_on;
    d.shift_inverse = fm.shift_inverse;
    d.shift_win = P.w_in;
    return d;
}

fht_status run_forward(const QuadPlan &P, const Side &image, const Side &out,
                       const FinalMap &fm, int t_lo, int t_hi, int acc_elem, void *ws,
                       cudaStream_t st) {
    for (int p = 0; p < P.npass; ++p) {
        PassDesc d = pass_desc(P, p, image, out, ws, fm, t_lo, t_hi);
        cudaError_t e = acc_elem == kF32 ? launch_pass<float>(P.m[p], d, false, st)
                                         : launch_pass<int32_t>(P.m[p], d, false, st);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

fht_status run_adjoint(const QuadPlan &P, const Side &grad_img, const Side &grad_hough,
                       const FinalMap &fm, int acc_elem, int accumulate, void *ws,
                       cudaStream_t st) {
    for (int p = P.npass - 1; p >= 0; --p) {
        PassDesc d = pass_desc(P, p, grad_img, grad_hough, ws, fm, 0, P.n - 1);
        d.accumulate = accumulate;
        cudaError_t e = acc_elem == kF32 ? launch_pass<float>(P.m[p], d, true, st)
                                         : launch_pass<int32_t>(P.m[p], d, true, st);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

bool sizes_ok(int h, int w) { return h >= 1 && w >= 1 && h <= kMaxSide && w <= kMaxSide; }
bool quadrant_ok(int q) { return q >= 0 && q <= 3; }

// fhtshift as a standalone permutation: one block row per Hough row.
struct ShiftRows {
    int layout;      // 0 quadrant, 1 full
    int q, n, hp, wp, W, w_in_q;
};

__device__ void row_quadrant(const ShiftRows &m, int r, int *q, int *t, int *w_in) {
    if (m.layout == 0) {
        *q = m.q; *t = r; *w_in = m.w_in_q;
        return;
    }
    int hp = m.hp, wp = m.wp;
    if (r < hp) { *q = 0; *t = hp - 1 - r; *w_in = wp; }
    else if (r < 2 * hp - 1) { *q = 1; *t = r - hp + 1; *w_in = wp; }
    else if (r < 2 * hp + wp - 2) { *q = 2; *t = 2 * hp + wp - 3 - r; *w_in = hp; }
    else { *q = 3; *t = r - 2 * hp - wp + 3; *w_in = hp; }
}

template <typename T>
__global__ void fhtshift_kernel(const T *in, T *out, int64_t in_pitch, int64_t out_pitch,
                                ShiftRows m, int inverse) {
    int r = blockIdx.x;
    int q, t, w_in;
    row_quadrant(m, r, &q, &t, &w_in);
    int sigma = (q == 0 || q == 3) ? 1 : -1;
    int s = fhtshift_amount(t, m.W, w_in, sigma);
    if (inverse) s = m.W - s;
    const T *src = in + (int64_t)r * in_pitch;
    T *dst = out + (int64_t)r * out_pitch;
    for (int x = threadIdx.x; x < m.W; x += blockDim.x) {
        int xo = x + s;
        if (xo >= m.W) xo -= m.W;
        dst[xo] = src[x];
    }
}

}  // namespace

// ============================================================== C ABI

extern "C" {

const char *fht_status_string(fht_status s) {
    switch (s) {
    case FHT_OK: return "ok";
    case FHT_EINVAL: return "invalid argument";
    case FHT_ENOMEM: return "out of memory";
    case FHT_ECUDA: return "CUDA error";
    case FHT_EUNSUPPORTED: return "unsupported";
    case FHT_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int fht_last_cuda_error(void) { return g_last_cuda_error; }

fht_status fht_query_shape(int h, int w, fht_quadrant q, int *rows, int *cols) {
    if (!sizes_ok(h, w) || !quadrant_ok(q) || !rows || !cols) return FHT_EINVAL;
    QuadPlan P = make_plan(h, w, q, false, kU8, kI32);
    *rows = P.n;
    *cols = P.W;
    return FHT_OK;
}

fht_status fht_full_shape(int h, int w, int *rows, int *cols) {
    if (!sizes_ok(h, w) || !rows || !cols) return FHT_EINVAL;
    int hp = next_pow2(h), wp = next_pow2(w);
    *rows = 2 * (hp + wp) - 3;
    *cols = hp + wp;
    return FHT_OK;
}

fht_status fht_full_row_to_quadrant(int h, int w, int row, int *q, int *t) {
    if (!sizes_ok(h, w) || !q || !t) return FHT_EINVAL;
    int hp = next_pow2(h), wp = next_pow2(w);
    if (row < 0 || row >= 2 * (hp + wp) - 3) return FHT_EINVAL;
    if (row < hp) { *q = 0; *t = hp - 1 - row; }
    else if (row < 2 * hp - 1) { *q = 1; *t = row - hp + 1; }
    else if (row < 2 * hp + wp - 2) { *q = 2; *t = 2 * hp + wp - 3 - row; }
    else { *q = 3; *t = row - 2 * hp - wp + 3; }
    return FHT_OK;
}

fht_status fht_angle_to_slopes(double phi_lo, double phi_hi, int h, int w, int *t_lo,
                               int *t_hi) {
    if (!sizes_ok(h, w) || !t_lo || !t_hi || !(phi_lo <= phi_hi)) return FHT_EINVAL;
    const double span_lo[4] = {-45.0, 0.0, 45.0, 90.0};
    const double span_hi[4] = {0.0, 45.0, 90.0, 135.0};
    const double deg = 3.14159265358979323846 / 180.0;
    for (int q = 0; q < 4; ++q) {
        t_lo[q] = t_hi[q] = -1;
        double a = std::max(phi_lo, span_lo[q]), b = std::min(phi_hi, span_hi[q]);
        if (a > b) continue;
        // angle measured away from the quadrant's slope-0 edge
        double th_a, th_b;
        switch (q) {
        case 0: th_a = -b; th_b = -a; break;
        case 1: th_a = a; th_b = b; break;
        case 2: th_a = 90.0 - b; th_b = 90.0 - a; break;
        default: th_a = a - 90.0; th_b = b - 90.0; break;
        }
        int n = next_pow2(q >= 2 ? w : h);
        int lo, hi;
        if (n == 1) {
            lo = hi = 0;
        } else {
            lo = (int)std::ceil((n - 1) * std::tan(th_a * deg) - 1e-9);
            hi = (int)std::floor((n - 1) * std::tan(th_b * deg) + 1e-9);
            lo = std::max(lo, 0);
            hi = std::min(hi, n - 1);
        }
        if (lo <= hi) { t_lo[q] = lo; t_hi[q] = hi; }
    }
    int n_h = next_pow2(h), n_w = next_pow2(w);
    if (t_lo[0] == 0 && t_lo[1] == 0) t_lo[1] = 1;
    if (t_hi[1] == n_h - 1 && t_hi[2] == n_w - 1) t_hi[2] = n_w - 2;
    if (t_lo[2] == 0 && t_lo[3] == 0) t_lo[3] = 1;
    for (int q = 0; q < 4; ++q)
        if (t_lo[q] > t_hi[q]) t_lo[q] = t_hi[q] = -1;
    return FHT_OK;
}

fht_status fht_workspace_size(int h, int w, fht_layout layout, fht_quadrant q,
                              fht_dtype in_t, fht_dtype acc_t, size_t *bytes) {
    if (!sizes_ok(h, w) || !bytes) return FHT_EINVAL;
    int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    size_t need = 0;
    if (layout == FHT_LAYOUT_FULL) {
        for (int qq = 0; qq < 4; ++qq)
            need = std::max(need, plan_workspace(make_plan(h, w, qq, true, elem_of(in_t), acc)));
    } else if (layout == FHT_LAYOUT_QUADRANT) {
        if (!quadrant_ok(q)) return FHT_EINVAL;
        need = plan_workspace(make_plan(h, w, q, false, elem_of(in_t), acc));
    } else {
        return FHT_EINVAL;
    }
    *bytes = need;
    return FHT_OK;
}

static fht_status forward_common(const void *img, fht_dtype in_t, int h, int w,
                                 int64_t in_pitch, fht_quadrant q, int t_lo, int t_hi,
                                 void *out, fht_dtype acc_t, int64_t out_pitch, void *ws,
                                 size_t ws_bytes, void *stream) {
    if (!img || !out || !sizes_ok(h, w) || !quadrant_ok(q) || in_pitch < w) return FHT_EINVAL;
    int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    QuadPlan P = make_plan(h, w, q, false, elem_of(in_t), acc);
    if (P.K > kMaxK) return FHT_EINVAL;
    if (t_lo < 0 || t_hi < t_lo || t_hi >= P.n) return FHT_EINVAL;
    if (out_pitch < P.W) return FHT_EINVAL;
    size_t need = plan_workspace(P);
    if (ws_bytes < need || (need > 0 && !ws)) return FHT_EINVAL;
    Side image{const_cast<void *>(img), in_pitch, elem_of(in_t), P.h_c, P.w_c};
    Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
    return run_forward(P, image, o, quadrant_map(t_lo, t_hi), t_lo, t_hi, acc, ws,
                       (cudaStream_t)stream);
}

fht_status fht_forward(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                       fht_quadrant q, void *out, fht_dtype acc_t, int64_t out_pitch,
                       void *workspace, size_t workspace_bytes, void *stream) {
    if (!sizes_ok(h, w) || !quadrant_ok(q)) return FHT_EINVAL;
    int n = next_pow2(q >= 2 ? w : h);
    return forward_common(img, in_t, h, w, in_pitch, q, 0, n - 1, out, acc_t, out_pitch,
                          workspace, workspace_bytes, stream);
}

fht_status fht_forward_range(const void *img, fht_dtype in_t, int h, int w,
                             int64_t in_pitch, fht_quadrant q, int t_lo, int t_hi,
                             void *out, fht_dtype acc_t, int64_t out_pitch,
                             void *workspace, size_t workspace_bytes, void *stream) {
    return forward_common(img, in_t, h, w, in_pitch, q, t_lo, t_hi, out, acc_t, out_pitch,
                          workspace, workspace_bytes, stream);
}

fht_status fht_full_quadrants(const void *img, fht_dtype in_t, int h, int w,
                              int64_t in_pitch, void *out, fht_dtype acc_t,
                              int64_t out_pitch, int apply_fhtshift, void *workspace,
                              size_t workspace_bytes, void *stream) {
    if (!img || !out || !sizes_ok(h, w) || in_pitch < w) return FHT_EINVAL;
    int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    int hp = next_pow2(h), wp = next_pow2(w);
    if (ilog2(hp) > kMaxK || ilog2(wp) > kMaxK) return FHT_EINVAL;
    if (out_pitch < hp + wp) return FHT_EINVAL;
    size_t need = 0;
    QuadPlan plans[4];
    for (int q = 0; q < 4; ++q) {
        plans[q] = make_plan(h, w, q, true, elem_of(in_t), acc);
        need = std::max(need, plan_workspace(plans[q]));
    }
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    for (int q = 0; q < 4; ++q) {
        const QuadPlan &P = plans[q];
        Side image{const_cast<void *>(img), in_pitch, elem_of(in_t), P.h_c, P.w_c};
        Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
        FinalMap fm = full_map(q, hp, wp);
        fm.shift_on = apply_fhtshift ? 1 : 0;
        fht_status s = run_forward(P, image, o, fm, fm.t_first, fm.t_last, acc, workspace,
                                   (cudaStream_t)stream);
        if (s != FHT_OK) return s;
    }
    return FHT_OK;
}

fht_status fhtshift(const void *in, void *out, fht_dtype dtype, int h, int w,
                    fht_layout layout, fht_quadrant q, int inverse, int64_t in_pitch,
                    int64_t out_pitch, void *stream) {
    if (!in || !out || !sizes_ok(h, w) || in == out) return FHT_EINVAL;
    if (dtype != FHT_I32 && dtype != FHT_F32) return FHT_EINVAL;
    ShiftRows m{};
    int rows;
    m.layout = layout == FHT_LAYOUT_FULL ? 1 : 0;
    m.hp = next_pow2(h);
    m.wp = next_pow2(w);
    if (layout == FHT_LAYOUT_FULL) {
        m.W = m.hp + m.wp;
        rows = 2 * m.W - 3;
    } else if (layout == FHT_LAYOUT_QUADRANT) {
        if (!quadrant_ok(q)) return FHT_EINVAL;
        QuadPlan P = make_plan(h, w, q, false, kU8, kI32);
        m.q = q;
        m.W = P.W;
        m.w_in_q = P.w_in;
        rows = P.n;
    } else {
        return FHT_EINVAL;
    }
    if (in_pitch < m.W || out_pitch < m.W) return FHT_EINVAL;
    dim3 grid(rows);
    cudaStream_t st = (cudaStream_t)stream;
    LaunchScope scope(dtype == FHT_I32 ? "fhtshift_i32" : "fhtshift_f32", st);
    if (dtype == FHT_I32)
        fhtshift_kernel<int32_t><<<grid, kBlock, 0, st>>>((const int32_t *)in, (int32_t *)out,
                                                          in_pitch, out_pitch, m, inverse);
    else
        fhtshift_kernel<float><<<grid, kBlock, 0, st>>>((const float *)in, (float *)out,
                                                        in_pitch, out_pitch, m, inverse);
    scope.done();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        return FHT_ECUDA;
    }
    return FHT_OK;
}

fht_status fht_adjoint(const void *grad_hough, fht_dtype dtype, int h, int w,
                       fht_layout layout, fht_quadrant q, int64_t in_pitch,
                       void *grad_img, int64_t out_pitch, void *workspace,
                       size_t workspace_bytes, void *stream) {
    if (!grad_hough || !grad_img || !sizes_ok(h, w) || out_pitch < w) return FHT_EINVAL;
    if (dtype != FHT_I32 && dtype != FHT_F32) return FHT_EINVAL;
    int acc = elem_of(dtype);
    cudaStream_t st = (cudaStream_t)stream;
    if (layout == FHT_LAYOUT_QUADRANT) {
        if (!quadrant_ok(q)) return FHT_EINVAL;
        QuadPlan P = make_plan(h, w, q, false, acc, acc);
        if (P.K > kMaxK || in_pitch < P.W) return FHT_EINVAL;
        size_t need = plan_workspace(P);
        if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
        Side gi{grad_img, out_pitch, acc, P.h_c, P.w_c};
        Side gh{const_cast<void *>(grad_hough), in_pitch, acc, 0, P.W};
        return run_adjoint(P, gi, gh, quadrant_map(0, P.n - 1), acc, 0, workspace, st);
    }
    if (layout != FHT_LAYOUT_FULL) return FHT_EINVAL;
    int hp = next_pow2(h), wp = next_pow2(w);
    if (ilog2(hp) > kMaxK || ilog2(wp) > kMaxK || in_pitch < hp + wp) return FHT_EINVAL;
    QuadPlan plans[4];
    size_t need = 0;
    for (int qq = 0; qq < 4; ++qq) {
        plans[qq] = make_plan(h, w, qq, true, acc, acc);
        need = std::max(need, plan_workspace(plans[qq]));
    }
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    for (int qq = 0; qq < 4; ++qq) {
        const QuadPlan &P = plans[qq];
        Side gi{grad_img, out_pitch, acc, P.h_c, P.w_c};
        Side gh{const_cast<void *>(grad_hough), in_pitch, acc, 0, P.W};
        fht_status s = run_adjoint(P, gi, gh, full_map(qq, hp, wp), acc, qq > 0 ? 1 : 0,
                                   workspace, st);
        if (s != FHT_OK) return s;
    }
    return FHT_OK;
}

fht_status fht_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_prof.clear();
    g_prof_on = true;
    return FHT_OK;
}

fht_status fht_profile_end(fht_kernel_time *out, int capacity, int *count) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_on = false;
        recs.swap(g_prof);
    }
    std::map<std::string, std::pair<int, double>> tot;
    fht_status st = FHT_OK;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            st = FHT_ECUDA;
        }
        auto &t = tot[r.name];
        t.first += 1;
        t.second += ms;
    }
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto &r : recs) {
            g_event_pool.push_back(r.a);
            g_event_pool.push_back(r.b);
        }
    }
    int i = 0;
    for (auto &kv : tot) {
        if (out && i < capacity) {
            snprintf(out[i].name, sizeof out[i].name, "%s", kv.first.c_str());
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    if (count) *count = i;
    return st;
}

long long fht_launch_count(void) { return g_launches.load(); }

}  // extern "C"
