// fht_api.cu -- C ABI (include/fht.h): argument checks, pass planning and
// kernel launches for the GB300 fast Hough transform.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fht.h"
#include "fht_host.h"
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
    double bytes;
};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

// Bytes taken off every destination span (fht_debug_test_hooks).
std::atomic<long long> g_debug_shrink{0};

// NVTX ranges per launch (FHT_NVTX=1 when the library loads).
const bool g_nvtx_on = [] {
    const char *e = getenv("FHT_NVTX");
    return e && e[0] == '1' && e[1] == 0;
}();

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

}  // namespace

namespace fht {

LaunchScope::LaunchScope(const char *name, cudaStream_t st, double alg_bytes)
    : st_(st), bytes_(alg_bytes) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_nvtx_on) {
        nvtxRangePushA(name);
        nvtx_ = true;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    on_ = g_prof_on;
    if (on_) {
        name_ = name;
        a_ = take_event();
        b_ = take_event();
        cudaEventRecord(a_, st_);
    }
}

void LaunchScope::done() {
    if (nvtx_) {
        nvtxRangePop();
        nvtx_ = false;
    }
    if (!on_) return;
    cudaEventRecord(b_, st_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(ProfRec{name_, a_, b_, bytes_});
    on_ = false;
}

}  // namespace fht

namespace {

constexpr int kBlock = 256;   // fhtshift kernel
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
int split_levels(int K, int *m, int max_levels = kMaxLevelsPerPass) {
    if (K == 0) { m[0] = 0; return 1; }
    int P = (K + max_levels - 1) / max_levels;
    for (int p = 0; p < P; ++p) m[p] = K / P + (p < K % P ? 1 : 0);
    return P;
}

// Tuning of the plain sum transforms and adjoints with 2^K rows: the most
// levels one pass fuses (stages per CTA) and the tile widths in warp-widths of
// source columns (first passes over uint8 images; passes with 4-byte shared
// tiles). Set by fht_set_tuning (an autotuner's results); defaults 6 levels
// and the FHT_TUNE widths.
struct TuneK {
    int max_levels, tile_u16, tile_wide;
};
TuneK tuning_for(int K);

// Geometry and pass plan of one quadrant transform.
struct QuadPlan {
    int q, sigma, transpose;
    bool adjoint;
    bool cyclic;        // every level all W columns wide, read cyclically
    int in_elem, acc_elem;
    int h_c, w_c;       // content size of the (transposed) image
    int n, K, W;
    int w_in;           // meaningful width used by fhtshift
    int npass;
    bool tuned;         // a plain sum transform or adjoint: the tuning table applies
    int m[4], k[5];
    int lvl_type[5];    // element type of intermediate level k[p] (1 <= p < npass)
    int lvl_cols[5];
    int64_t lvl_pitch[5];
    size_t buf_bytes[2];
    // adjoint: the level the final pass reads is windowed when win_len > 0
    // (PassDesc::lo_win / hi_win)
    int win_len, win_c;
};

// Plan of quadrant q. With `adjoint`, the plan is the transform's transpose:
// the opposite-sign transform of the gradient (the dyadic offsets are
// symmetric in slope and row), every level all W columns wide and cyclic.
// With `sheared`, the quadrant's own transform of the sheared image (Section
// 4), also on cyclic full-width levels: the shear moves the black zone, so
// the compact columns do not hold. w_scaled > 0 replaces the content width
// (columns of the (transposed) image) by that of its scaled rows (Section 4).
// n_rows > 0 pads the (transposed) image to that many rows instead of the
// next power of two of its height, and W_cols > 0 sets the cyclic width (a
// strip of a sharded image is transformed with the whole image's n_s rows
// and width).
QuadPlan make_plan(int h, int w, int q, bool full, int in_elem, int acc_elem,
                   bool adjoint = false, bool sheared = false, int op = 0, int w_scaled = 0,
                   int n_rows = 0, int W_cols = 0) {
    QuadPlan P{};
    P.q = q;
    P.adjoint = adjoint;
    P.cyclic = adjoint || sheared;
    P.in_elem = in_elem;
    P.acc_elem = acc_elem;
    P.transpose = q >= 2;
    P.sigma = (q == 0 || q == 3) ? 1 : -1;
    if (adjoint) P.sigma = -P.sigma;
    P.h_c = P.transpose ? w : h;
    P.w_c = P.transpose ? h : w;
    if (w_scaled > 0) P.w_c = w_scaled;
    P.n = n_rows > 0 ? n_rows : next_pow2(P.h_c);
    P.K = ilog2(P.n);
    if (full) {
        P.W = next_pow2(h) + next_pow2(w);
        P.w_in = P.W - P.n;
    } else {
        P.W = P.w_c + P.n;
        P.w_in = P.w_c;
    }
    if (W_cols > 0) P.W = W_cols;
    P.tuned = op == 0 && !sheared;
    P.npass = split_levels(P.K, P.m, P.tuned ? tuning_for(P.K).max_levels : kMaxLevelsPerPass);
    P.k[0] = 0;
    for (int p = 0; p < P.npass; ++p) P.k[p + 1] = P.k[p] + P.m[p];
    P.buf_bytes[0] = P.buf_bytes[1] = 0;
    P.win_len = P.win_c = 0;
    if (adjoint && P.npass >= 2)
        adjoint_window(P.w_c, P.W, P.K, P.m[P.npass - 1], P.sigma, &P.win_len, &P.win_c);
    for (int p = 1; p < P.npass; ++p) {
        int k = P.k[p];
        int type = acc_elem;
        // u8 images summed over 2^k rows stay below 2^16 while k <= 8 (the
        // sum's passes from a uint16 level write int32: only the first level)
        if (acc_elem == kI32 && in_elem == kU8 && k <= 8 && !adjoint && (p == 1 || op != 0))
            type = kU16;
        // the maximum or minimum of uint8 values is one of them: uint16 at every level
        if (acc_elem == kI32 && in_elem == kU8 && op != 0) type = kU16;
        P.lvl_type[p] = type;
        P.lvl_cols[p] = P.cyclic ? P.W : std::min(P.W, P.w_c + (1 << k));
        P.lvl_pitch[p] = (int64_t)align_up(P.lvl_cols[p], 64);
        if (P.win_len > 0 && p == P.npass - 1) {
            // windowed: loads of 8 from any index below win_len stay in the row
            P.lvl_cols[p] = P.win_len;
            P.lvl_pitch[p] = (int64_t)align_up((size_t)P.win_len + 16, 64);
        }
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

// Pick the fused-kernel instantiation for the pass's element types. Shared
// tiles of a first pass over a uint8 image hold level-3 values (<= 255*8) as
// uint16.
cudaError_t launch_forward(int M, const PassDesc &d, int acc, cudaStream_t st) {
    const int src = d.lo.type, dst = d.hi.type;
    if (acc == kF32) {
        if (src == kU8) return launch_fused_f32_u8(M, d, st);
        return launch_fused_f32_f32(M, d, st);
    }
    if (src == kU8) {
        if (dst == kU16) return launch_fused_i32_u8_u16(M, d, st);
        return launch_fused_i32_u8_i32(M, d, st);
    }
    if (src == kU16) return launch_fused_i32_u16(M, d, st);
    return launch_fused_i32_i32(M, d, st);
}

// The same for the maximum (op 1) or minimum (op 2) along the patterns:
// uint8 images keep uint16 levels throughout.
cudaError_t launch_forward_op(int M, const PassDesc &d, int acc, int op, cudaStream_t st) {
    const int src = d.lo.type, dst = d.hi.type;
    const bool mx = op == 1;
    if (acc == kF32) return mx ? launch_max_f32(M, d, st) : launch_min_f32(M, d, st);
    if (src == kU8) {
        if (dst == kU16) return mx ? launch_max_i32_u8_u16(M, d, st) : launch_min_i32_u8_u16(M, d, st);
        return mx ? launch_max_i32_u8_i32(M, d, st) : launch_min_i32_u8_i32(M, d, st);
    }
    if (dst == kU16) return mx ? launch_max_i32_u16_u16(M, d, st) : launch_min_i32_u16_u16(M, d, st);
    return mx ? launch_max_i32_u16_i32(M, d, st) : launch_min_i32_u16_i32(M, d, st);
}

// Block-A warp-columns per tile: wider tiles compute less halo but need more
// shared memory (fewer CTAs per SM). Overridable for tuning through
// FHT_TUNE="n_a_u16,n_a_wide".
struct Tune {
    int n_a_u16 = 1;    // first pass over uint8 images (uint16 shared tile)
    int n_a_wide = 1;   // 4-byte shared tiles
    bool staged = true;
    bool concurrent = true;
    Tune() {
        if (const char *e = getenv("FHT_TUNE")) {
            int a = 0, b = 0;
            if (sscanf(e, "%d,%d", &a, &b) == 2 && a >= 1 && a <= 3 && b >= 1 && b <= 3) {
                n_a_u16 = a;
                n_a_wide = b;
            }
        }
        if (const char *e = getenv("FHT_STAGED")) staged = !(e[0] == '0' && e[1] == 0);
        if (const char *e = getenv("FHT_CONCURRENT")) concurrent = !(e[0] == '0' && e[1] == 0);
    }
};
const Tune g_tune;

// The tuning table (index K = 1..15), guarded by g_tune_mu; entries never set
// hold the defaults.
constexpr int kTuneSlots = 16;
std::mutex g_tune_mu;
TuneK g_tune_k[kTuneSlots];
bool g_tune_set[kTuneSlots] = {};

TuneK tuning_for(int K) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (K >= 0 && K < kTuneSlots && g_tune_set[K]) return g_tune_k[K];
    return TuneK{kMaxLevelsPerPass, g_tune.n_a_u16, g_tune.n_a_wide};
}

std::mutex &counter_mu() {
    static std::mutex mu;
    return mu;
}
std::vector<unsigned int (*)()> &counter_fns() {
    static std::vector<unsigned int (*)()> fns;
    return fns;
}

}  // namespace

namespace fht {

bool staged_enabled() { return g_tune.staged; }

long long debug_hi_shrink() { return g_debug_shrink.load(); }

bool register_device_counter(unsigned int (*read_and_reset)()) {
    std::lock_guard<std::mutex> lk(counter_mu());
    counter_fns().push_back(read_and_reset);
    return true;
}

unsigned int read_device_counters() {
    std::lock_guard<std::mutex> lk(counter_mu());
    unsigned int n = 0;
    for (auto f : counter_fns()) n += f();
    return n;
}

}  // namespace fht

namespace {

// First passes over uint8 images keep their shared tile in uint16.
bool acc_is_u16_mid(const QuadPlan &P, int p) { return p == 0 && P.in_elem == kU8 && P.acc_elem == kI32; }

// A uniform batch of same-size transforms: image b's source, destination and
// workspace lie b * src / dst / ws bytes past image 0's.
struct Batch {
    int count = 1;
    int64_t src = 0, dst = 0, ws = 0;
};

PassDesc pass_desc(const QuadPlan &P, int p, const Side &image, const Side &final_side,
                   void *ws, const FinalMap &fm, int t_lo, int t_hi, const Batch &B = Batch{}) {
    PassDesc d{};
    d.batch = B.count;
    d.lo_bstride = p == 0 ? B.src : B.ws;
    d.hi_bstride = p == P.npass - 1 ? B.dst : B.ws;
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
    const int drop1 = P.K - P.k[p + 1];
    d.need_lo = t_lo >> drop1;
    d.need_hi = t_hi >> drop1;
    d.s_count = P.n >> P.k[p + 1];
    d.p_begin = 0;
    d.p_count = d.hi.cols;
    d.cyclic = P.cyclic ? 1 : 0;
    d.t_first = fm.t_first;
    d.t_last = fm.t_last;
    d.row_base = fm.row_base;
    d.row_dir = fm.row_dir;
    d.shift_on = fm.shift_on;
    d.shift_inverse = fm.shift_inverse;
    d.shift_win = P.w_in;
    d.black_wc = P.w_c;
    // block A has 2^MB items per warp-column: widen it until every warp has one
    if (P.m[p] >= 4) {
        const int rb = 1 << (P.m[p] - 3);
        const TuneK t = P.tuned ? tuning_for(P.K) : TuneK{kMaxLevelsPerPass, g_tune.n_a_u16,
                                                            g_tune.n_a_wide};
        const int base = acc_is_u16_mid(P, p) ? t.tile_u16 : t.tile_wide;
        d.n_a = std::max(base, 8 / rb);
    } else {
        d.n_a = 1;
    }
    return d;
}

fht_status run_forward(const QuadPlan &P, const Side &image, const Side &out,
                       const FinalMap &fm, int t_lo, int t_hi, int acc_elem, void *ws,
                       cudaStream_t st, const Batch &B = Batch{}, bool range_call = false) {
    for (int p = 0; p < P.npass; ++p) {
        PassDesc d = pass_desc(P, p, image, out, ws, fm, t_lo, t_hi, B);
        d.range_call = range_call ? 1 : 0;
        cudaError_t e = launch_forward(P.m[p], d, acc_elem, st);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

// Transpose of quadrant plan P (built with adjoint = true): the gradient's
// rows t come from grad_hough through `fm`; the result is cropped to the
// (transposed) image and written, or added, into grad_img.
fht_status run_adjoint(const QuadPlan &P, const Side &grad_img, const Side &grad_hough,
                       const FinalMap &fm, int acc_elem, int accumulate, void *ws,
                       cudaStream_t st, const Batch &B = Batch{},
                       cudaEvent_t before_final = nullptr) {
    for (int p = 0; p < P.npass; ++p) {
        if (before_final && p == P.npass - 1) {
            // the final pass adds into an image gradient another stream writes
            const cudaError_t e = cudaStreamWaitEvent(st, before_final, 0);
            if (e != cudaSuccess) {
                g_last_cuda_error = (int)e;
                return FHT_ECUDA;
            }
        }
        // output rows y < h_c of the opposite-sign transform are the image rows
        PassDesc d = pass_desc(P, p, grad_hough, grad_img, ws, FinalMap{0, P.n - 1, 0, 1, 0, 0},
                               0, P.h_c - 1, B);
        if (p == 0) {
            d.transpose = 0;
            d.lo.cols = P.W;
            d.src_t_first = fm.t_first;
            d.src_t_last = fm.t_last;
            d.src_row_base = fm.row_base;
            d.src_row_dir = fm.row_dir;
        }
        d.win_len = P.win_len;
        d.win_c = P.win_c;
        if (P.win_len > 0) {
            d.lo_win = p == P.npass - 1;
            d.hi_win = p == P.npass - 2;
            if (d.hi_win) {
                // the pass still covers every column; its stores keep the windows
                d.hi.cols = P.W;
                d.p_count = P.W;
            }
        }
        if (d.hi_final) {
            d.dst_image = 1;
            d.dst_h = P.h_c;
            d.dst_w = P.w_c;
            d.dst_transpose = P.transpose;
            d.accumulate = accumulate;
            d.hi.cols = P.W;
            // only columns X < w_c reach the image: p = X + sigma_plus * n
            d.p_begin = P.sigma > 0 ? P.n : 0;
            d.p_count = P.w_c;
        }
        cudaError_t e = acc_elem == kF32 ? launch_adjoint_f32(P.m[p], d, st)
                                         : launch_adjoint_i32(P.m[p], d, st);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

bool sizes_ok(int h, int w) { return h >= 1 && w >= 1 && h <= kMaxSide && w <= kMaxSide; }
bool quadrant_ok(int q) { return q >= 0 && q <= 3; }

// ------------------------------------------------------------ concurrent quadrants
// The four quadrants of a full transform are independent: the forward writes
// disjoint rows of the full image, and the adjoint's passes before the final
// one read disjoint rows of the gradient. Given a workspace slice each, they
// run on four streams -- the caller's and three of the library's, forked from
// and joined back into the caller's stream with events, which stream capture
// turns into graph branches -- so one quadrant's launch tails overlap
// another's work. The adjoint's final passes all add into the one image
// gradient, so they stay in quadrant order (an event chain). Each device has
// kForkSets sets of streams, taken by successive calls in turn, so that calls
// the caller runs concurrently on its own streams do not queue behind each
// other on the library's; a mutex keeps each call's fork-join sequence whole.
// The streams and events are created by the first call on a device that is
// not being captured; a call captured before then runs its quadrants one
// after another. While per-launch profiling is on, quadrants also run one
// after another so that every launch is timed alone.
constexpr int kForkDevices = 64;
constexpr int kForkSets = 4;
struct ForkState {
    cudaStream_t lane[3] = {};
    cudaEvent_t fork = nullptr, join[3] = {}, chain[4] = {};
};
std::mutex g_fork_mu;
ForkState g_fork[kForkDevices][kForkSets];
bool g_fork_ready[kForkDevices] = {};
unsigned g_fork_next[kForkDevices] = {};

bool profiling_on() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof_on;
}

bool use_concurrent(size_t ws_bytes, size_t concurrent_bytes) {
    return g_tune.concurrent && concurrent_bytes > 0 && ws_bytes >= concurrent_bytes &&
           !profiling_on();
}

class QuadFork {
  public:
    explicit QuadFork(cudaStream_t st) : st_(st), lk_(g_fork_mu) {}
    // Sets up this device's streams and events on first use, then makes the
    // library's streams wait for the work already on the caller's stream.
    // FHT_EUNSUPPORTED (nothing enqueued): the streams do not exist yet and
    // the caller's stream is being captured; run the quadrants serially.
    fht_status begin() {
        int dev = -1;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess || dev < 0 || dev >= kForkDevices) return fail(e);
        if (!g_fork_ready[dev]) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if ((e = cudaStreamIsCapturing(st_, &cs)) != cudaSuccess) return fail(e);
            if (cs != cudaStreamCaptureStatusNone) return FHT_EUNSUPPORTED;
            const unsigned fl = cudaEventDisableTiming;
            for (int k = 0; k < kForkSets && e == cudaSuccess; ++k) {
                ForkState &S = g_fork[dev][k];
                for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                    e = cudaStreamCreateWithFlags(&S.lane[i], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.fork, fl);
                for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                    e = cudaEventCreateWithFlags(&S.join[i], fl);
                for (int i = 0; i < 4 && e == cudaSuccess; ++i)
                    e = cudaEventCreateWithFlags(&S.chain[i], fl);
            }
            if (e != cudaSuccess) return fail(e);
            g_fork_ready[dev] = true;
        }
        F_ = &g_fork[dev][g_fork_next[dev]++ % kForkSets];
        if ((e = cudaEventRecord(F_->fork, st_)) != cudaSuccess) return fail(e);
        for (int i = 0; i < 3; ++i) {
            if ((e = cudaStreamWaitEvent(F_->lane[i], F_->fork, 0)) != cudaSuccess) return fail(e);
            forked_ = i + 1;
        }
        return FHT_OK;
    }
    cudaStream_t stream(int q) const { return q == 0 ? st_ : F_->lane[q - 1]; }
    cudaEvent_t chain(int q) const { return F_->chain[q]; }
    // Joins every forked stream back into the caller's stream (also after a
    // failed launch: a capture must not end with a stream left out).
    fht_status end() {
        fht_status s = FHT_OK;
        for (int i = 0; i < forked_; ++i) {
            cudaError_t e = cudaEventRecord(F_->join[i], F_->lane[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st_, F_->join[i], 0);
            if (e != cudaSuccess) s = fail(e);
        }
        forked_ = 0;
        return s;
    }
    ~QuadFork() { end(); }

  private:
    static fht_status fail(cudaError_t e) {
        g_last_cuda_error = (int)(e != cudaSuccess ? e : cudaErrorInvalidDevice);
        return FHT_ECUDA;
    }
    cudaStream_t st_;
    std::lock_guard<std::mutex> lk_;
    ForkState *F_ = nullptr;
    int forked_ = 0;
};

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

// Rotates rows of 4-byte words: out[r][(x + s_r) mod W] = in[r][x]. One
// group of `lanes` threads (a power of two, 32..kBlock) per row.
//
// Vector path (W and both pitches multiples of 4 words, both bases 16-byte
// aligned): each thread writes aligned 16-byte output vectors. Output words
// 4j..4j+3 come from source words x0..x0+3 (mod W), x0 = 4j - s (mod W); as W
// is a multiple of 4 the row's wrap falls between aligned vectors, so those
// words lie in the aligned source vectors a and a+1 (mod W/4), at the offset
// o = (-s) mod 4, which is the same for the whole row.
__global__ void __launch_bounds__(kBlock)
    fhtshift_kernel(const uint32_t *in, uint32_t *out, int64_t in_pitch, int64_t out_pitch,
                    ShiftRows m, int inverse, int rows, int lanes_log2, int vec) {
    const int lanes = 1 << lanes_log2;
    const int lane = threadIdx.x & (lanes - 1);
    const int r = blockIdx.x * (kBlock >> lanes_log2) + (threadIdx.x >> lanes_log2);
    if (r >= rows) return;
    int q, t, w_in;
    row_quadrant(m, r, &q, &t, &w_in);
    const int sigma = (q == 0 || q == 3) ? 1 : -1;
    int s = fhtshift_amount(t, m.W, w_in, sigma);   // in [0, W)
    if (inverse) s = m.W - s;                         // in (0, W]
    if (vec) {
        const int nv = m.W >> 2;
        const uint4 *src = reinterpret_cast<const uint4 *>(in + (int64_t)r * in_pitch);
        uint4 *dst = reinterpret_cast<uint4 *>(out + (int64_t)r * out_pitch);
        const int o = (-s) & 3;
        const int sv = (s + o) >> 2;   // x0 = 4 (j - sv) + o, sv in [0, nv]
#pragma unroll 4
        for (int j = lane; j < nv; j += lanes) {
            int a = j - sv;
            if (a < 0) a += nv;
            const uint4 v0 = __ldg(src + a);
            uint4 res = v0;
            if (o != 0) {
                const uint4 v1 = __ldg(src + (a + 1 == nv ? 0 : a + 1));
                if (o == 1) res = make_uint4(v0.y, v0.z, v0.w, v1.x);
                else if (o == 2) res = make_uint4(v0.z, v0.w, v1.x, v1.y);
                else res = make_uint4(v0.w, v1.x, v1.y, v1.z);
            }
            dst[j] = res;
        }
        return;
    }
    const uint32_t *src = in + (int64_t)r * in_pitch;
    uint32_t *dst = out + (int64_t)r * out_pitch;
    for (int x = lane; x < m.W; x += lanes) {
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
    case FHT_EBOUNDS: return "access outside a pass's buffers (debug build)";
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
    // the adjoint of an (acc, acc) transform runs full-width intermediates
    const bool adj = in_t == acc_t;
    if (layout == FHT_LAYOUT_FULL) {
        // one slice per quadrant, so that the quadrants can run concurrently
        for (int qq = 0; qq < 4; ++qq) {
            size_t one = plan_workspace(make_plan(h, w, qq, true, elem_of(in_t), acc));
            if (adj) one = std::max(one, plan_workspace(make_plan(h, w, qq, true, acc, acc, true)));
            need += one;
        }
    } else if (layout == FHT_LAYOUT_QUADRANT) {
        if (!quadrant_ok(q)) return FHT_EINVAL;
        need = plan_workspace(make_plan(h, w, q, false, elem_of(in_t), acc));
        if (adj) need = std::max(need, plan_workspace(make_plan(h, w, q, false, acc, acc, true)));
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
                       (cudaStream_t)stream, Batch{}, t_lo != 0 || t_hi != P.n - 1);
}

// ------------------------------------------------------------ strips of a sharded image

// Rows (h_c) and columns (w_c) of the (transposed) strip, and whether n and W
// fit it: n a power of two >= h_c (up to 2^kMaxK), W >= w_c + n.
static bool padded_ok(int h, int w, fht_quadrant q, int n, int W, int *h_c, int *w_c) {
    if (!quadrant_ok(q) || h < 0 || w < 0 || h > kMaxSide || w > kMaxSide) return false;
    *h_c = q >= 2 ? w : h;
    *w_c = q >= 2 ? h : w;
    if (*w_c < 1 || n < 1 || (n & (n - 1)) != 0 || ilog2(n) > kMaxK || n < *h_c) return false;
    return W >= *w_c + n && W <= 2 * kMaxSide;
}

fht_status fht_workspace_size_padded(int h, int w, fht_quadrant q, int n, int W, fht_dtype in_t,
                                     fht_dtype acc_t, size_t *bytes) {
    int h_c = 0, w_c = 0;
    if (!bytes || !padded_ok(h, w, q, n, W, &h_c, &w_c)) return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    *bytes = h_c == 0 ? 0
                      : plan_workspace(make_plan(h, w, q, false, elem_of(in_t), acc, false,
                                                 false, 0, 0, n, W));
    return FHT_OK;
}

fht_status fht_forward_padded(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                              fht_quadrant q, int n, int W, void *out, fht_dtype acc_t,
                              int64_t out_pitch, void *workspace, size_t workspace_bytes,
                              void *stream) {
    int h_c = 0, w_c = 0;
    if (!out || !padded_ok(h, w, q, n, W, &h_c, &w_c) || out_pitch < W) return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    if (h_c == 0) {
        // an empty strip: every level, and so the result, is zero
        const cudaError_t e = cudaMemset2DAsync(out, (size_t)out_pitch * 4, 0, (size_t)W * 4, n,
                                                (cudaStream_t)stream);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
        return FHT_OK;
    }
    if (!img || in_pitch < w) return FHT_EINVAL;
    QuadPlan P = make_plan(h, w, q, false, elem_of(in_t), acc, false, false, 0, 0, n, W);
    const size_t need = plan_workspace(P);
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    Side image{const_cast<void *>(img), in_pitch, elem_of(in_t), P.h_c, P.w_c};
    Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
    return run_forward(P, image, o, quadrant_map(0, P.n - 1), 0, P.n - 1, acc, workspace,
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
    size_t need = 0, sum = 0;
    QuadPlan plans[4];
    for (int q = 0; q < 4; ++q) {
        plans[q] = make_plan(h, w, q, true, elem_of(in_t), acc);
        need = std::max(need, plan_workspace(plans[q]));
        sum += plan_workspace(plans[q]);
    }
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    auto run_q = [&](int q, void *ws, cudaStream_t st) {
        const QuadPlan &P = plans[q];
        Side image{const_cast<void *>(img), in_pitch, elem_of(in_t), P.h_c, P.w_c};
        Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
        FinalMap fm = full_map(q, hp, wp);
        fm.shift_on = apply_fhtshift ? 1 : 0;
        return run_forward(P, image, o, fm, fm.t_first, fm.t_last, acc, ws, st);
    };
    if (use_concurrent(workspace_bytes, sum)) {
        QuadFork f((cudaStream_t)stream);
        fht_status s = f.begin();
        if (s != FHT_EUNSUPPORTED) {
            char *ws = static_cast<char *>(workspace);
            for (int q = 0; q < 4 && s == FHT_OK; ++q) {
                s = run_q(q, ws, f.stream(q));
                ws += plan_workspace(plans[q]);
            }
            const fht_status j = f.end();
            return s != FHT_OK ? s : j;
        }
    }
    for (int q = 0; q < 4; ++q) {
        fht_status s = run_q(q, workspace, (cudaStream_t)stream);
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
    const bool vec = m.W % 4 == 0 && in_pitch % 4 == 0 && out_pitch % 4 == 0 &&
                     reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 16 == 0;
    const int units = vec ? m.W / 4 : m.W;   // per row, one thread each
    int lanes_log2 = 5;
    while ((1 << lanes_log2) < units && (1 << lanes_log2) < kBlock) ++lanes_log2;
    const int rows_per_block = kBlock >> lanes_log2;
    dim3 grid((rows + rows_per_block - 1) / rows_per_block);
    cudaStream_t st = (cudaStream_t)stream;
    LaunchScope scope(dtype == FHT_I32 ? "fhtshift_i32" : "fhtshift_f32", st,
                      2.0 * rows * m.W * 4.0);
    // both types are moved as 4-byte words
    fhtshift_kernel<<<grid, kBlock, 0, st>>>(static_cast<const uint32_t *>(in),
                                             static_cast<uint32_t *>(out), in_pitch, out_pitch,
                                             m, inverse, rows, lanes_log2, vec ? 1 : 0);
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
        QuadPlan P = make_plan(h, w, q, false, acc, acc, true);
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
    size_t need = 0, sum = 0;
    for (int qq = 0; qq < 4; ++qq) {
        plans[qq] = make_plan(h, w, qq, true, acc, acc, true);
        need = std::max(need, plan_workspace(plans[qq]));
        sum += plan_workspace(plans[qq]);
    }
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    auto run_q = [&](int qq, void *ws, cudaStream_t s_q, cudaEvent_t before_final) {
        const QuadPlan &P = plans[qq];
        Side gi{grad_img, out_pitch, acc, P.h_c, P.w_c};
        Side gh{const_cast<void *>(grad_hough), in_pitch, acc, 0, P.W};
        return run_adjoint(P, gi, gh, full_map(qq, hp, wp), acc, qq > 0 ? 1 : 0, ws, s_q,
                           Batch{}, before_final);
    };
    if (use_concurrent(workspace_bytes, sum)) {
        // quadrant qq's final pass waits for quadrant qq-1's (event chain)
        QuadFork f(st);
        fht_status s = f.begin();
        if (s != FHT_EUNSUPPORTED) {
            char *ws = static_cast<char *>(workspace);
            for (int qq = 0; qq < 4 && s == FHT_OK; ++qq) {
                s = run_q(qq, ws, f.stream(qq), qq > 0 ? f.chain(qq - 1) : nullptr);
                if (s == FHT_OK) {
                    const cudaError_t e = cudaEventRecord(f.chain(qq), f.stream(qq));
                    if (e != cudaSuccess) {
                        g_last_cuda_error = (int)e;
                        s = FHT_ECUDA;
                    }
                }
                ws += plan_workspace(plans[qq]);
            }
            const fht_status j = f.end();
            return s != FHT_OK ? s : j;
        }
    }
    for (int qq = 0; qq < 4; ++qq) {
        fht_status s = run_q(qq, workspace, st, nullptr);
        if (s != FHT_OK) return s;
    }
    return FHT_OK;
}

// ------------------------------------------------------------ other operations

fht_status fht_forward_op(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                          fht_quadrant q, fht_op op, int t_lo, int t_hi, void *out,
                          fht_dtype acc_t, int64_t out_pitch, void *workspace,
                          size_t workspace_bytes, void *stream) {
    if (op == FHT_OP_SUM)
        return forward_common(img, in_t, h, w, in_pitch, q, t_lo, t_hi, out, acc_t, out_pitch,
                              workspace, workspace_bytes, stream);
    if (op != FHT_OP_MAX && op != FHT_OP_MIN) return FHT_EINVAL;
    if (!img || !out || !sizes_ok(h, w) || !quadrant_ok(q) || in_pitch < w) return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    const bool u8_i32 = in_t == FHT_U8 && acc_t == FHT_I32;
    const bool f32_f32 = in_t == FHT_F32 && acc_t == FHT_F32;
    if (!u8_i32 && !f32_f32) return FHT_EUNSUPPORTED;
    QuadPlan P = make_plan(h, w, q, false, elem_of(in_t), acc, false, false, (int)op);
    if (P.K > kMaxK) return FHT_EINVAL;
    if (t_lo < 0 || t_hi < t_lo || t_hi >= P.n || out_pitch < P.W) return FHT_EINVAL;
    const size_t need = plan_workspace(P);
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    Side image{const_cast<void *>(img), in_pitch, elem_of(in_t), P.h_c, P.w_c};
    Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
    for (int p = 0; p < P.npass; ++p) {
        PassDesc d = pass_desc(P, p, image, o, workspace, quadrant_map(t_lo, t_hi), t_lo, t_hi);
        d.range_call = t_lo != 0 || t_hi != P.n - 1;
        const cudaError_t e = launch_forward_op(P.m[p], d, acc, (int)op, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

// ------------------------------------------------------------ sheared (Section 4)

static bool spl_ok(double spl) { return spl >= -1.0 && spl <= 1.0; }   // false for NaN

fht_status fht_workspace_size_sheared(int h, int w, fht_quadrant q, fht_dtype in_t,
                                      fht_dtype acc_t, size_t *bytes) {
    if (!sizes_ok(h, w) || !quadrant_ok(q) || !bytes) return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    *bytes = plan_workspace(make_plan(h, w, q, false, elem_of(in_t), acc, false, true));
    return FHT_OK;
}

// The sheared forward transform of Section 4 on the cyclic pass code: every
// pass carries the shear in fixed point (shear_p); P was built with sheared =
// true (for the scaled transform, on the scaled width, img being the scaled
// copy).
static fht_status run_sheared(const QuadPlan &P, const void *img, int in_elem, int64_t in_pitch,
                              long long shear_p, int t_lo, int t_hi, void *out, fht_dtype acc_t,
                              int64_t out_pitch, void *workspace, cudaStream_t st) {
    const int acc = P.acc_elem;
    Side image{const_cast<void *>(img), in_pitch, in_elem, P.h_c, P.w_c};
    Side o{out, out_pitch, elem_of(acc_t), 0, P.W};
    for (int p = 0; p < P.npass; ++p) {
        PassDesc d = pass_desc(P, p, image, o, workspace, quadrant_map(t_lo, t_hi), t_lo, t_hi);
        d.shear_on = 1;
        d.shear_p = shear_p;
        if (d.hi_final) {
            // every column X of the slope rows [t_lo, t_hi]: p = X + sigma_plus * n
            d.dst_image = 1;
            d.dst_row_lo = t_lo;
            d.dst_h = t_hi + 1;
            d.dst_w = P.W;
            d.dst_transpose = 0;
            d.accumulate = 0;
            d.hi.cols = P.W;
            d.p_begin = P.sigma > 0 ? P.n : 0;
            d.p_count = P.W;
        }
        // cyclic pass code for the pass's element types (a uint8 image's
        // first level is uint16, as in the compact forward)
        cudaError_t e;
        if (acc == kF32)
            e = d.lo.type == kU8 ? launch_adjoint_f32_u8(P.m[p], d, st)
                                 : launch_adjoint_f32(P.m[p], d, st);
        else if (d.lo.type == kU8)
            e = d.hi.type == kU16 ? launch_adjoint_i32_u8_u16(P.m[p], d, st)
                                  : launch_adjoint_i32_u8(P.m[p], d, st);
        else if (d.lo.type == kU16)
            e = launch_adjoint_i32_u16(P.m[p], d, st);
        else
            e = launch_adjoint_i32(P.m[p], d, st);
        if (e != cudaSuccess) {
            g_last_cuda_error = (int)e;
            return FHT_ECUDA;
        }
    }
    return FHT_OK;
}

// spl in fixed point, 32 fractional bits, rounded half up (exact in double
// for |spl| <= 1)
static long long shear_fixed(double spl) { return (long long)std::floor(spl * 4294967296.0 + 0.5); }

fht_status fht_forward_sheared(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                               fht_quadrant q, double spl, int t_lo, int t_hi, void *out,
                               fht_dtype acc_t, int64_t out_pitch, void *workspace,
                               size_t workspace_bytes, void *stream) {
    if (!img || !out || !sizes_ok(h, w) || !quadrant_ok(q) || in_pitch < w || !spl_ok(spl))
        return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    const int in_elem = elem_of(in_t);
    QuadPlan P = make_plan(h, w, q, false, in_elem, acc, false, true);
    if (P.K > kMaxK) return FHT_EINVAL;
    if (t_lo < 0 || t_hi < t_lo || t_hi >= P.n || out_pitch < P.W) return FHT_EINVAL;
    const size_t need = plan_workspace(P);
    if (workspace_bytes < need || (need > 0 && !workspace)) return FHT_EINVAL;
    return run_sheared(P, img, in_elem, in_pitch, shear_fixed(spl), t_lo, t_hi, out, acc_t,
                       out_pitch, workspace, (cudaStream_t)stream);
}

// ------------------------------------------------------------ scaled (Section 4)

static bool alpha_ok(double alpha) { return alpha >= 1.0 / 256.0 && alpha <= 256.0; }

// Source step D = ceil(2^32 / alpha) and scaled width ceil(w * 2^32 / D) of
// a row of w pixels; false when the scaled row is empty or wider than the
// library's largest side.
static bool scaled_geometry(int w, double alpha, long long *step, int *w_alpha) {
    if (!alpha_ok(alpha) || w < 1) return false;
    const long long D = (long long)std::ceil(4294967296.0 / alpha);
    const long long wa = (((long long)w << 32) + D - 1) / D;
    if (D < 1 || wa < 1 || wa > kMaxSide) return false;
    *step = D;
    *w_alpha = (int)wa;
    return true;
}

fht_status fht_scaled_width(int w, double alpha, int *w_alpha) {
    long long D = 0;
    if (!w_alpha || w > kMaxSide || !scaled_geometry(w, alpha, &D, w_alpha)) return FHT_EINVAL;
    return FHT_OK;
}

fht_status fht_scaled_shape(int h, int w, fht_quadrant q, double alpha, int *rows, int *cols) {
    if (!rows || !cols || !sizes_ok(h, w) || !quadrant_ok(q)) return FHT_EINVAL;
    long long D = 0;
    int wa = 0;
    if (!scaled_geometry(q >= 2 ? h : w, alpha, &D, &wa)) return FHT_EINVAL;
    *rows = next_pow2(q >= 2 ? w : h);
    *cols = wa + *rows;
    return FHT_OK;
}

// The scaled copy of the image the scaled transform reads, placed in the
// workspace after the plan's level buffers: Q0/Q1 scale every image row to
// w_alpha columns (h x w_alpha), Q2/Q3 the image's row index (w_alpha x w
// rows, read transposed); rows padded to 16 bytes.
struct ScaledCopy {
    bool along_rows;
    int rows, cols;
    int64_t pitch;   // elements
    size_t offset, bytes;
};

static ScaledCopy scaled_copy(const QuadPlan &P, int h, int w, fht_quadrant q, int wa,
                              int in_elem) {
    ScaledCopy c;
    const int eb = (int)elem_bytes(in_elem);
    c.along_rows = q >= 2;
    c.rows = c.along_rows ? wa : h;
    c.cols = c.along_rows ? w : wa;
    const int g = 16 / eb;
    c.pitch = ((int64_t)c.cols + g - 1) / g * g;
    c.offset = (plan_workspace(P) + 255) / 256 * 256;
    c.bytes = (size_t)c.rows * (size_t)c.pitch * (size_t)eb;
    return c;
}

fht_status fht_workspace_size_scaled(int h, int w, fht_quadrant q, double alpha, fht_dtype in_t,
                                     fht_dtype acc_t, size_t *bytes) {
    if (!sizes_ok(h, w) || !quadrant_ok(q) || !bytes) return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    long long D = 0;
    int wa = 0;
    if (!scaled_geometry(q >= 2 ? h : w, alpha, &D, &wa)) return FHT_EINVAL;
    const QuadPlan P = make_plan(h, w, q, false, elem_of(in_t), acc, false, true, 0, wa);
    const ScaledCopy c = scaled_copy(P, h, w, q, wa, elem_of(in_t));
    *bytes = c.offset + c.bytes;
    return FHT_OK;
}

fht_status fht_forward_scaled(const void *img, fht_dtype in_t, int h, int w, int64_t in_pitch,
                              fht_quadrant q, double alpha, double spl, int t_lo, int t_hi,
                              void *out, fht_dtype acc_t, int64_t out_pitch, void *workspace,
                              size_t workspace_bytes, void *stream) {
    if (!img || !out || !sizes_ok(h, w) || !quadrant_ok(q) || in_pitch < w || !spl_ok(spl))
        return FHT_EINVAL;
    const int acc = acc_kind(in_t, acc_t);
    if (acc < 0) return FHT_EINVAL;
    long long D = 0;
    int wa = 0;
    if (!scaled_geometry(q >= 2 ? h : w, alpha, &D, &wa)) return FHT_EINVAL;
    const int in_elem = elem_of(in_t);
    QuadPlan P = make_plan(h, w, q, false, in_elem, acc, false, true, 0, wa);
    if (P.K > kMaxK) return FHT_EINVAL;
    if (t_lo < 0 || t_hi < t_lo || t_hi >= P.n || out_pitch < P.W) return FHT_EINVAL;
    const ScaledCopy c = scaled_copy(P, h, w, q, wa, in_elem);
    if (!workspace || workspace_bytes < c.offset + c.bytes) return FHT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    void *copy = static_cast<char *>(workspace) + c.offset;
    const cudaError_t e = launch_scale_image(img, in_pitch, (int)elem_bytes(in_elem), c.along_rows,
                                             D, copy, c.pitch, c.rows, c.cols, st);
    if (e != cudaSuccess) {
        g_last_cuda_error = (int)e;
        return FHT_ECUDA;
    }
    return run_sheared(P, copy, in_elem, c.pitch, shear_fixed(spl), t_lo, t_hi, out, acc_t,
                       out_pitch, workspace, st);
}

fht_status fht_scale_range(double phi_lo, double phi_hi, int h, int w, fht_quadrant *q,
                           double *alpha, double *spl, int *t_lo, int *t_hi) {
    if (!q || !alpha || !spl || !t_lo || !t_hi || !sizes_ok(h, w) || !(phi_lo <= phi_hi))
        return FHT_EINVAL;
    const double rad = M_PI / 180.0;
    const double mid = 0.5 * (phi_lo + phi_hi);
    int qq;
    double a, b, edge;
    if (mid >= -45.0 && mid <= 45.0 && phi_lo > -90.0 && phi_hi < 90.0) {
        qq = FHT_Q0;
        a = phi_lo;
        b = phi_hi;
        edge = std::tan(b * rad);
    } else if (mid > 45.0 && mid <= 135.0 && phi_lo > 0.0 && phi_hi < 180.0) {
        qq = FHT_Q3;
        a = phi_lo - 90.0;
        b = phi_hi - 90.0;
        edge = std::tan(a * rad);
    } else {
        return FHT_EINVAL;
    }
    const double span = std::tan(b * rad) - std::tan(a * rad);
    double al = 16.0;
    if (span > 0) al = std::min(al, 1.0 / span);
    if (edge != 0) al = std::min(al, 1.0 / std::fabs(edge));
    int rows = 0, cols = 0;
    fht_query_shape(h, w, (fht_quadrant)qq, &rows, &cols);
    int hi = 0;
    if (rows > 1) hi = std::min(rows - 1, (int)std::floor((rows - 1) * al * span + 1e-9));
    *q = (fht_quadrant)qq;
    *alpha = al;
    *spl = qq == FHT_Q0 ? al * edge : -al * edge;
    *t_lo = 0;
    *t_hi = hi;
    return FHT_OK;
}

fht_status fht_shear_range(double phi_lo, double phi_hi, int h, int w, fht_quadrant *q,
                           double *spl, int *t_lo, int *t_hi) {
    if (!q || !spl || !t_lo || !t_hi || !sizes_ok(h, w) || !(phi_lo <= phi_hi))
        return FHT_EINVAL;
    const double rad = M_PI / 180.0;
    int qq;
    double a, b, s;
    if (phi_lo >= -45.0 && phi_hi <= 45.0) {
        qq = FHT_Q0;
        a = phi_lo;
        b = phi_hi;
        s = std::tan(b * rad);
    } else if (phi_lo >= 45.0 && phi_hi <= 135.0) {
        qq = FHT_Q3;
        a = phi_lo - 90.0;
        b = phi_hi - 90.0;
        s = -std::tan(a * rad);
    } else {
        return FHT_EINVAL;
    }
    const double span = std::tan(b * rad) - std::tan(a * rad);
    if (span > 1.0 + 1e-12) return FHT_EINVAL;
    int rows = 0, cols = 0;
    fht_query_shape(h, w, (fht_quadrant)qq, &rows, &cols);
    int hi = 0;
    if (rows > 1) hi = std::min(rows - 1, (int)std::floor((rows - 1) * span + 1e-9));
    *q = (fht_quadrant)qq;
    *spl = s;
    *t_lo = 0;
    *t_hi = hi;
    return FHT_OK;
}

// ------------------------------------------------------------ uniform batches

// Workspace of one image of a uniform FP32 batch: the forward's and the
// adjoint's intermediate levels, rounded to 256 bytes.
static fht_status many_image_ws(int h, int w, fht_layout layout, fht_quadrant q, size_t *bytes) {
    size_t one = 0;
    const fht_status s = fht_workspace_size(h, w, layout, q, FHT_F32, FHT_F32, &one);
    if (s != FHT_OK) return s;
    *bytes = (one + 255) / 256 * 256;
    return FHT_OK;
}

static bool many_args_ok(int batch, int h, int w, fht_layout layout, fht_quadrant q) {
    if (batch < 1 || batch > 65535 || !sizes_ok(h, w)) return false;
    if (layout == FHT_LAYOUT_QUADRANT) return quadrant_ok(q);
    return layout == FHT_LAYOUT_FULL;
}

fht_status fht_workspace_size_many(int batch, int h, int w, fht_layout layout, fht_quadrant q,
                                   size_t *bytes) {
    if (!bytes || !many_args_ok(batch, h, w, layout, q)) return FHT_EINVAL;
    size_t one = 0;
    const fht_status s = many_image_ws(h, w, layout, q, &one);
    if (s != FHT_OK) return s;
    *bytes = one * (size_t)batch;
    return FHT_OK;
}

fht_status fht_forward_many(const void *img, int batch, int64_t img_batch_stride, int h, int w,
                            int64_t in_pitch, fht_layout layout, fht_quadrant q, void *out,
                            int64_t out_batch_stride, int64_t out_pitch, void *workspace,
                            size_t workspace_bytes, void *stream) {
    if (!img || !out || !many_args_ok(batch, h, w, layout, q) || in_pitch < w) return FHT_EINVAL;
    int rows = 0, cols = 0;
    const fht_status sq = layout == FHT_LAYOUT_FULL ? fht_full_shape(h, w, &rows, &cols)
                                                    : fht_query_shape(h, w, q, &rows, &cols);
    if (sq != FHT_OK || out_pitch < cols) return FHT_EINVAL;
    // images and outputs of the batch must not overlap one another
    if (batch > 1 && (img_batch_stride < (int64_t)h * in_pitch ||
                      out_batch_stride < (int64_t)rows * out_pitch))
        return FHT_EINVAL;
    size_t one = 0;
    fht_status s = many_image_ws(h, w, layout, q, &one);
    if (s != FHT_OK) return s;
    if (workspace_bytes < one * (size_t)batch || (one > 0 && !workspace)) return FHT_EINVAL;
    Batch B;
    B.count = batch;
    B.src = img_batch_stride * 4;
    B.dst = out_batch_stride * 4;
    B.ws = (int64_t)one;
    cudaStream_t st = (cudaStream_t)stream;
    if (layout == FHT_LAYOUT_QUADRANT) {
        QuadPlan P = make_plan(h, w, q, false, kF32, kF32);
        if (P.K > kMaxK) return FHT_EINVAL;
        Side image{const_cast<void *>(img), in_pitch, kF32, P.h_c, P.w_c};
        Side o{out, out_pitch, kF32, 0, P.W};
        return run_forward(P, image, o, quadrant_map(0, P.n - 1), 0, P.n - 1, kF32, workspace,
                           st, B);
    }
    const int hp = next_pow2(h), wp = next_pow2(w);
    if (ilog2(hp) > kMaxK || ilog2(wp) > kMaxK) return FHT_EINVAL;
    for (int qq = 0; qq < 4; ++qq) {
        QuadPlan P = make_plan(h, w, qq, true, kF32, kF32);
        Side image{const_cast<void *>(img), in_pitch, kF32, P.h_c, P.w_c};
        Side o{out, out_pitch, kF32, 0, P.W};
        const FinalMap fm = full_map(qq, hp, wp);
        s = run_forward(P, image, o, fm, fm.t_first, fm.t_last, kF32, workspace, st, B);
        if (s != FHT_OK) return s;
    }
    return FHT_OK;
}

fht_status fht_adjoint_many(const void *grad_hough, int batch, int64_t grad_batch_stride, int h,
                            int w, fht_layout layout, fht_quadrant q, int64_t in_pitch,
                            void *grad_img, int64_t img_batch_stride, int64_t out_pitch,
                            void *workspace, size_t workspace_bytes, void *stream) {
    if (!grad_hough || !grad_img || !many_args_ok(batch, h, w, layout, q) || out_pitch < w)
        return FHT_EINVAL;
    int rows = 0, cols = 0;
    const fht_status sq = layout == FHT_LAYOUT_FULL ? fht_full_shape(h, w, &rows, &cols)
                                                    : fht_query_shape(h, w, q, &rows, &cols);
    if (sq != FHT_OK || in_pitch < cols) return FHT_EINVAL;
    if (batch > 1 && (grad_batch_stride < (int64_t)rows * in_pitch ||
                      img_batch_stride < (int64_t)h * out_pitch))
        return FHT_EINVAL;
    size_t one = 0;
    fht_status s = many_image_ws(h, w, layout, q, &one);
    if (s != FHT_OK) return s;
    if (workspace_bytes < one * (size_t)batch || (one > 0 && !workspace)) return FHT_EINVAL;
    Batch B;
    B.count = batch;
    B.src = grad_batch_stride * 4;
    B.dst = img_batch_stride * 4;
    B.ws = (int64_t)one;
    cudaStream_t st = (cudaStream_t)stream;
    if (layout == FHT_LAYOUT_QUADRANT) {
        QuadPlan P = make_plan(h, w, q, false, kF32, kF32, true);
        if (P.K > kMaxK) return FHT_EINVAL;
        Side gi{grad_img, out_pitch, kF32, P.h_c, P.w_c};
        Side gh{const_cast<void *>(grad_hough), in_pitch, kF32, 0, P.W};
        return run_adjoint(P, gi, gh, quadrant_map(0, P.n - 1), kF32, 0, workspace, st, B);
    }
    const int hp = next_pow2(h), wp = next_pow2(w);
    if (ilog2(hp) > kMaxK || ilog2(wp) > kMaxK) return FHT_EINVAL;
    for (int qq = 0; qq < 4; ++qq) {
        QuadPlan P = make_plan(h, w, qq, true, kF32, kF32, true);
        Side gi{grad_img, out_pitch, kF32, P.h_c, P.w_c};
        Side gh{const_cast<void *>(grad_hough), in_pitch, kF32, 0, P.W};
        s = run_adjoint(P, gi, gh, full_map(qq, hp, wp), kF32, qq > 0 ? 1 : 0, workspace, st, B);
        if (s != FHT_OK) return s;
    }
    return FHT_OK;
}

fht_status fht_set_tuning(int K, const fht_tuning *t) {
    if (K < 1 || K > kMaxK) return FHT_EINVAL;
    if (t && (t->max_levels < 4 || t->max_levels > kMaxLevelsPerPass || t->tile_u8 < 1 ||
              t->tile_u8 > 3 || t->tile_wide < 1 || t->tile_wide > 3))
        return FHT_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (t) g_tune_k[K] = TuneK{t->max_levels, t->tile_u8, t->tile_wide};
    g_tune_set[K] = t != nullptr;
    return FHT_OK;
}

fht_status fht_get_tuning(int K, fht_tuning *out) {
    if (K < 1 || K > kMaxK || !out) return FHT_EINVAL;
    const TuneK t = tuning_for(K);
    out->max_levels = t.max_levels;
    out->tile_u8 = t.tile_u16;
    out->tile_wide = t.tile_wide;
    return FHT_OK;
}

fht_status fht_device_status(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        g_last_cuda_error = (int)cudaGetLastError();
        return FHT_ECUDA;
    }
    return read_device_counters() ? FHT_EBOUNDS : FHT_OK;
}

fht_status fht_debug_test_hooks(long long shrink_bytes) {
#ifdef FHT_DEBUG
    if (shrink_bytes < 0) return FHT_EINVAL;
    g_debug_shrink.store(shrink_bytes);
    return FHT_OK;
#else
    (void)shrink_bytes;
    return FHT_EUNSUPPORTED;
#endif
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
    struct Tot {
        int launches = 0;
        double ms = 0, bytes = 0;
    };
    std::map<std::string, Tot> tot;
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
        t.launches += 1;
        t.ms += ms;
        t.bytes += r.bytes;
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
            out[i].launches = kv.second.launches;
            out[i].total_ms = kv.second.ms;
            out[i].alg_bytes = kv.second.bytes;
        }
        ++i;
    }
    if (count) *count = i;
    return st;
}

long long fht_launch_count(void) { return g_launches.load(); }

}  // extern "C"
