// fht_batched.cu -- many images of different sizes in one persistent launch.
//
// Each image gets its own quadrant plan (padded to its own power of two, one
// or two passes). The plan lists work "segments" (image, pass), ordered by
// pass, then kernel variant, then image; every segment holds groups x tiles
// items. Persistent CTAs take items in that order from a global counter. An
// item of pass p > 0 waits until all items of pass p - 1 of its image are
// done; since items are taken in order and every taken item belongs to a
// running CTA that never waits on a later item, the waits always end. Each
// wait is still bounded by a clock budget: past it the CTA records
// FHT_ETIMEOUT and skips the item, so the launch always ends.
// Float plans carry a second work list, the adjoints (the transpose of every
// image's quadrant), launched the same way by fht_adjoint_batched.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/fht.h"
#include "fht_batched.cuh"
#include "fht_host.h"

using namespace fht;
using namespace fht::batched;

// Direct launches of one table stage it in turn in this many pinned copies,
// so the host can run that many launches ahead.
constexpr int kDirectTables = 3;

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// The batched tuning in force (fht_set_batched_tuning), read at plan creation.
std::mutex g_btune_mu;
fht_batched_tuning default_batched_tuning() {
    fht_batched_tuning t{};
    t.units_per_item = 4;
    t.tile_u8 = 2;
    t.tile_wide = 1;
    t.ctas_per_sm = 2;
    return t;
}
fht_batched_tuning g_btune = default_batched_tuning();

bool batched_tuning_ok(const fht_batched_tuning &t) {
    if (t.units_per_item < 1 || t.units_per_item > 16) return false;
    if (t.tile_u8 < 1 || t.tile_u8 > 3 || t.tile_wide < 1 || t.tile_wide > 3) return false;
    if (t.ctas_per_sm != 2 && t.ctas_per_sm != 3) return false;
    for (int K = 7; K <= kMaxBatchK; ++K) {
        const int f = t.first_levels[K];
        if (f != 0 && (f < K - 6 || f > 6)) return false;
    }
    return true;
}

// One launchable work list (the forward transforms, or the adjoints, of the
// batch) and its pinned staging. Workspace layout of a launch: the segment
// table at 0, the counters at counters_off, the per-(image, pass) done
// counters at done_off, the intermediate levels from levels_off.
struct Table {
    int n_segs = 0, total_items = 0, n_done = 0;
    size_t table_bytes = 0, counters_off = 0, done_off = 0, levels_off = 0;
    size_t ws_bytes = 0, smem = 0;
    // kDirectTables copies used in turn by direct launches (each reused only
    // once its previous copy has run); the segments as built, without
    // pointers, follow them (the template a capture's own table starts from)
    void *host_table = nullptr;
    cudaEvent_t copied[kDirectTables] = {};
    bool copy_pending[kDirectTables] = {};
    int next_table = 0;
    // one pinned table per stream capture, kept until the plan is destroyed:
    // a captured graph's copy node reads its own table at every replay, so a
    // later capture (or direct call) never changes what an earlier graph runs
    std::vector<void *> capture_tables;
};

void release_table(Table &T) {
    for (int c = 0; c < kDirectTables; ++c) {
        if (!T.copied[c]) continue;
        if (T.copy_pending[c]) cudaEventSynchronize(T.copied[c]);
        cudaEventDestroy(T.copied[c]);
        T.copied[c] = nullptr;
    }
    if (T.host_table) cudaFreeHost(T.host_table);
    T.host_table = nullptr;
    for (void *p : T.capture_tables) cudaFreeHost(p);
    T.capture_tables.clear();
}

// A new pinned table for a stream capture, copied from the template. The
// capture is in progress on this thread: the allocation (no stream work) is
// made in the relaxed capture mode, which lets it proceed without ending the
// capture, and the caller's mode is restored afterwards.
void *new_capture_table(Table &T) {
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    if (cudaThreadExchangeStreamCaptureMode(&mode) != cudaSuccess) return nullptr;
    void *p = nullptr;
    const cudaError_t e = cudaMallocHost(&p, T.counters_off);
    cudaThreadExchangeStreamCaptureMode(&mode);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    try {
        T.capture_tables.push_back(p);
    } catch (...) {
        cudaFreeHost(p);
        return nullptr;
    }
    std::memcpy(p, static_cast<unsigned char *>(T.host_table) + kDirectTables * T.counters_off,
                T.table_bytes);
    return p;
}

}  // namespace

struct fht_plan {
    int count = 0;
    int f32 = 0;
    int q = 0;
    int sigma = 1;
    Table fwd, adj;
    bool has_adj = false;   // float plans also carry the adjoints' table
    size_t ws_bytes = 0;
    std::vector<int> h, w, rows, cols;   // per image: size, and its quadrant's n x W
    long long wait_budget = 4000000000LL;   // ~2 s of SM clocks
    int dep_bias = 0;
    int minb = 2;   // CTAs per SM of the kernel instantiation (tuning at creation)
    size_t last_counters_off = 0;   // counters of the table launched last
};

namespace {

// Segments of every image's passes, ordered by pass, variant, m, image.
// adjoint: the transpose of each image's quadrant (float only), computed
// as in fht_adjoint: the opposite-sign transform of the gradient with cyclic
// full-width levels, the final level cropped into the image gradient.
fht_status build_table(const int *hs, const int *ws, int count, fht_quadrant q, bool f32,
                       bool adjoint, const fht_batched_tuning &tun, Table &T) {
    const bool u8 = !f32;
    std::vector<BatchSeg> segs;
    size_t level_bytes = 0, smem = 0;
    int n_done = 0;
    struct Pending {
        BatchSeg s;
        int pass;
    };
    std::vector<Pending> pend;
    for (int j = 0; j < count; ++j) {
        int rows = 0, cols = 0;
        if (fht_query_shape(hs[j], ws[j], q, &rows, &cols) != FHT_OK) return FHT_EINVAL;
        int K = 0;
        while ((1 << K) < rows) ++K;
        if (K > kMaxBatchK) return FHT_EUNSUPPORTED;
        const int transpose = q >= 2;
        const int sigma_q = (q == 0 || q == 3) ? 1 : -1;
        const int sigma = adjoint ? -sigma_q : sigma_q;
        const int h_c = transpose ? ws[j] : hs[j], w_c = transpose ? hs[j] : ws[j];
        const int n = rows, W = cols;
        int ms[2], npass;
        if (K <= 6) {
            ms[0] = K;
            npass = 1;
        } else {
            // the tuning's split, else as even as possible (first pass larger)
            ms[0] = tun.first_levels[K] ? tun.first_levels[K] : (K + 1) / 2;
            ms[1] = K - ms[0];
            npass = 2;
        }
        // the one intermediate level (after pass 0): uint16 for uint8 images;
        // compact columns for forward transforms, all W (cyclic) for adjoints
        size_t lvl_off = 0;
        int lvl_cols = 0;
        int64_t lvl_pitch = 0;
        const int lvl_type = f32 ? kF32 : kU16;
        int win_len = 0, win_c = 0;
        if (npass == 2) {
            lvl_cols = adjoint ? W : std::min(W, w_c + (1 << ms[0]));
            lvl_pitch = (lvl_cols + 63) / 64 * 64;
            if (adjoint) {
                // the level the final pass reads keeps each row's window only
                adjoint_window(w_c, W, K, ms[1], sigma, &win_len, &win_c);
                if (win_len > 0) {
                    lvl_cols = win_len;
                    lvl_pitch = (win_len + 16 + 63) / 64 * 64;
                }
            }
            lvl_off = level_bytes;
            level_bytes += align256((size_t)n * lvl_pitch * (f32 ? 4 : 2));
        }
        int prev_items = 0;
        for (int p = 0; p < npass; ++p) {
            const int m = ms[p], k0 = p == 0 ? 0 : ms[0], k1 = k0 + m;
            BatchSeg s{};
            PassDesc &d = s.d;
            d.lo_image = p == 0;
            d.transpose = adjoint ? 0 : transpose;
            d.hi_final = p == npass - 1;
            d.n = n;
            d.W = W;
            d.K = K;
            d.k0 = k0;
            d.sigma = sigma;
            d.s_count = n >> k1;
            d.t_first = 0;
            d.t_last = n - 1;
            d.row_base = 0;
            d.row_dir = 1;
            d.shift_win = w_c;
            d.black_wc = w_c;
            if (!adjoint) {
                d.a_lo = 0;
                d.a_count = 1 << k0;
                d.need_lo = 0;
                d.need_hi = (1 << k1) - 1;
                d.lo = p == 0 ? Side{nullptr, 0, f32 ? kF32 : kU8, h_c, w_c}
                              : Side{nullptr, lvl_pitch, lvl_type, n, lvl_cols};
                d.hi = d.hi_final ? Side{nullptr, 0, f32 ? kF32 : kI32, 0, W}
                                  : Side{nullptr, lvl_pitch, lvl_type, n, lvl_cols};
                d.p_begin = 0;
                d.p_count = d.hi.cols;
            } else {
                // output rows y < h_c of the opposite-sign transform are the
                // image rows: only the slopes they depend on are computed
                d.a_lo = 0;
                d.a_count = ((h_c - 1) >> (K - k0)) + 1;
                d.need_lo = 0;
                d.need_hi = (h_c - 1) >> (K - k1);
                d.cyclic = 1;
                d.win_len = win_len;
                d.win_c = win_c;
                d.lo_win = win_len > 0 && p == 1;
                d.hi_win = win_len > 0 && p == 0;
                if (p == 0) {
                    d.lo = Side{nullptr, 0, kF32, n, W};
                    d.src_t_first = 0;
                    d.src_t_last = n - 1;
                    d.src_row_base = 0;
                    d.src_row_dir = 1;
                } else {
                    d.lo = Side{nullptr, lvl_pitch, kF32, n, lvl_cols};
                }
                if (d.hi_final) {
                    d.hi = Side{nullptr, 0, kF32, h_c, W};
                    d.dst_image = 1;
                    d.dst_h = h_c;
                    d.dst_w = w_c;
                    d.dst_transpose = transpose;
                    d.accumulate = 0;
                    // only columns X < w_c reach the image: p = X + sigma_plus * n
                    d.p_begin = sigma > 0 ? n : 0;
                    d.p_count = w_c;
                } else {
                    d.hi = Side{nullptr, lvl_pitch, kF32, n, W};
                    d.p_begin = 0;
                    d.p_count = W;
                }
            }
            const bool u16_mid = u8 && p == 0;
            if (m >= 4) {
                // block A has 2^(m-3) items per warp-column: widen the tile
                // until every warp has one
                const int rb = 1 << (m - 3);
                d.n_a = std::max(u16_mid ? tun.tile_u8 : tun.tile_wide, 8 / rb);
            } else {
                d.n_a = 1;
            }
            const int MA = m <= 3 ? m : 3, MB = m - MA;
            const int pad = u16_mid ? 2 : 1;
            const TileGeom G = tile_geom(MA, MB, d.n_a, kWarps, pad);
            d.tile_w = G.tile_out;
            d.tiles = (d.p_count + G.tile_out - 1) / G.tile_out;
            if (MB > 0)
                smem = std::max(smem, (size_t)(1 << m) * G.pitch * (u16_mid ? 2 : 4));
            s.m = m;
            s.image = j;
            s.variant = f32 ? kVarF32 : (p == 0 ? (npass == 1 ? kVarU8Final : kVarU8Level)
                                                : kVarU16Final);
            s.tiles = d.tiles;
            s.units = d.s_count * d.a_count * d.tiles;
            s.chunk = std::max(1, std::min(tun.units_per_item, s.units));
            s.lo_from_image = p == 0;
            s.hi_from_image = d.hi_final;
            s.lo_off = (int64_t)lvl_off;
            s.hi_off = (int64_t)lvl_off;
            s.done_index = n_done + p;
            s.dep_index = p == 0 ? -1 : n_done + p - 1;
            s.dep_count = prev_items;
            prev_items = (s.units + s.chunk - 1) / s.chunk;
            pend.push_back(Pending{s, p});
        }
        n_done += npass;
    }
    // order: pass, variant, m, image
    std::stable_sort(pend.begin(), pend.end(), [](const Pending &x, const Pending &y) {
        if (x.pass != y.pass) return x.pass < y.pass;
        if (x.s.variant != y.s.variant) return x.s.variant < y.s.variant;
        return x.s.m < y.s.m;
    });
    int items = 0;
    for (auto &pd : pend) {
        pd.s.item_begin = items;
        items += (pd.s.units + pd.s.chunk - 1) / pd.s.chunk;
        segs.push_back(pd.s);
    }
    T.n_segs = (int)segs.size();
    T.total_items = items;
    T.n_done = n_done;
    T.smem = smem;
    T.table_bytes = segs.size() * sizeof(BatchSeg);
    T.counters_off = align256(T.table_bytes);
    T.done_off = T.counters_off + 256;
    T.levels_off = align256(T.done_off + (size_t)n_done * sizeof(unsigned int));
    // intermediate offsets inside the workspace
    for (auto &s : segs) {
        s.lo_off += (int64_t)T.levels_off;
        s.hi_off += (int64_t)T.levels_off;
    }
    T.ws_bytes = T.levels_off + level_bytes;
    if (cudaMallocHost(&T.host_table, (kDirectTables + 1) * T.counters_off) != cudaSuccess) {
        cudaGetLastError();
        T.host_table = nullptr;
        return FHT_ENOMEM;
    }
    for (int c = 0; c < kDirectTables; ++c) {
        if (cudaEventCreateWithFlags(&T.copied[c], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            T.copied[c] = nullptr;
            return FHT_ECUDA;
        }
    }
    for (int c = 0; c <= kDirectTables; ++c)
        std::memcpy(static_cast<unsigned char *>(T.host_table) + c * T.counters_off,
                    segs.data(), T.table_bytes);
    return FHT_OK;
}

// Stage table T with the call's pointers (src/dst per image, from the
// caller's descriptors), copy it and clear the counters on the stream, and
// launch kernel k over it.
struct CallPtrs {
    const void *src;
    int64_t src_pitch;
    void *dst;
    int64_t dst_pitch;
};

fht_status launch_table(fht_plan *plan, Table &T, const CallPtrs *calls, Kernel k,
                        const char *name, void *workspace, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FHT_ECUDA;
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    // a direct launch takes the next table of the ring, once the copy of the
    // launch that used it last has read it; a capture gets a table of its own
    const int tab = T.next_table;
    unsigned char *table = nullptr;
    if (capturing) {
        table = static_cast<unsigned char *>(new_capture_table(T));
        if (!table) return FHT_ENOMEM;
    } else {
        T.next_table = (T.next_table + 1) % kDirectTables;
        if (T.copy_pending[tab]) {
            if (cudaEventSynchronize(T.copied[tab]) != cudaSuccess) return FHT_ECUDA;
            T.copy_pending[tab] = false;
        }
        table = static_cast<unsigned char *>(T.host_table) + (size_t)tab * T.counters_off;
    }
    BatchSeg *segs = reinterpret_cast<BatchSeg *>(table);
    for (int i = 0; i < T.n_segs; ++i) {
        BatchSeg &sg = segs[i];
        const CallPtrs &c = calls[sg.image];
        if (sg.lo_from_image) {
            sg.d.lo.ptr = const_cast<void *>(c.src);
            sg.d.lo.pitch = c.src_pitch;
        } else {
            sg.d.lo.ptr = ws + sg.lo_off;
        }
        if (sg.hi_from_image) {
            sg.d.hi.ptr = c.dst;
            sg.d.hi.pitch = c.dst_pitch;
        } else {
            sg.d.hi.ptr = ws + sg.hi_off;
        }
        set_debug_extents(sg.d);
    }
    cudaError_t e = cudaMemcpyAsync(ws, table, T.counters_off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !capturing) {
        e = cudaEventRecord(T.copied[tab], st);
        if (e == cudaSuccess) T.copy_pending[tab] = true;
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ws + T.counters_off, 0, T.levels_off - T.counters_off, st);
    if (e != cudaSuccess) return FHT_ECUDA;
    if (T.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T.smem);
        if (e != cudaSuccess) return FHT_ECUDA;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, T.smem);
    int grid = std::max(1, sms * std::max(per_sm, 1));
    grid = std::min(grid, std::max(T.total_items, 1));
    plan->last_counters_off = T.counters_off;
    LaunchScope scope(name, st, 0.0);
    k<<<grid, kWarps * 32, T.smem, st>>>(
        reinterpret_cast<const BatchSeg *>(ws), T.n_segs, T.total_items,
        reinterpret_cast<Counters *>(ws + T.counters_off),
        reinterpret_cast<unsigned int *>(ws + T.done_off), plan->wait_budget, plan->dep_bias);
    scope.done();
    e = cudaGetLastError();
    return e == cudaSuccess ? FHT_OK : FHT_ECUDA;
}

}  // namespace

extern "C" {

fht_status fht_plan_create_batched(const int *hs, const int *ws, int count, fht_quadrant q,
                                   fht_dtype in_t, fht_dtype acc_t, fht_plan **plan,
                                   size_t *workspace_bytes) {
    if (!hs || !ws || !plan || !workspace_bytes || count <= 0 || q < 0 || q > 3)
        return FHT_EINVAL;
    const bool f32 = acc_t == FHT_F32 && in_t == FHT_F32;
    const bool u8 = acc_t == FHT_I32 && in_t == FHT_U8;
    if (!f32 && !u8) return FHT_EUNSUPPORTED;
    for (int j = 0; j < count; ++j) {
        int r = 0, c = 0;
        if (fht_query_shape(hs[j], ws[j], q, &r, &c) != FHT_OK) return FHT_EINVAL;
        if (r > (1 << kMaxBatchK)) return FHT_EUNSUPPORTED;
    }
    fht_batched_tuning tun;
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        tun = g_btune;
    }
    fht_plan *P = new (std::nothrow) fht_plan();
    if (!P) return FHT_ENOMEM;
    P->count = count;
    P->f32 = f32;
    P->q = q;
    P->sigma = (q == 0 || q == 3) ? 1 : -1;
    P->minb = tun.ctas_per_sm;
    fht_status s = build_table(hs, ws, count, q, f32, false, tun, P->fwd);
    if (s == FHT_OK && f32) {
        s = build_table(hs, ws, count, q, true, true, tun, P->adj);
        P->has_adj = s == FHT_OK;
    }
    if (s != FHT_OK) {
        fht_plan_destroy(P);
        return s;
    }
    P->ws_bytes = std::max(P->fwd.ws_bytes, P->has_adj ? P->adj.ws_bytes : 0);
    for (int j = 0; j < count; ++j) {
        int r = 0, c = 0;
        fht_query_shape(hs[j], ws[j], q, &r, &c);
        P->h.push_back(hs[j]);
        P->w.push_back(ws[j]);
        P->rows.push_back(r);
        P->cols.push_back(c);
    }
    *plan = P;
    *workspace_bytes = P->ws_bytes;
    return FHT_OK;
}

fht_status fht_forward_batched(fht_plan *plan, const fht_image_desc *descs, void *workspace,
                               size_t workspace_bytes, void *stream) {
    if (!plan || !descs || !workspace || workspace_bytes < plan->ws_bytes) return FHT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return FHT_EINVAL;
    std::vector<CallPtrs> calls(plan->count);
    for (int j = 0; j < plan->count; ++j) {
        const fht_image_desc &dj = descs[j];
        if (!dj.img || !dj.out || dj.img_pitch < plan->w[j] || dj.out_pitch < plan->cols[j])
            return FHT_EINVAL;
        calls[j] = CallPtrs{dj.img, dj.img_pitch, dj.out, dj.out_pitch};
    }
    const int mb = plan->minb;
    const Kernel k = plan->f32 ? (plan->sigma > 0 ? kernel_f32_pos(mb) : kernel_f32_neg(mb))
                               : (plan->sigma > 0 ? kernel_u8_pos(mb) : kernel_u8_neg(mb));
    return launch_table(plan, plan->fwd, calls.data(), k,
                        plan->f32 ? "batched_forward_f32" : "batched_forward_u8_i32", workspace,
                        stream);
}

fht_status fht_adjoint_batched(fht_plan *plan, const fht_adjoint_desc *descs, void *workspace,
                               size_t workspace_bytes, void *stream) {
    if (!plan || !descs || !workspace || workspace_bytes < plan->ws_bytes) return FHT_EINVAL;
    if (!plan->has_adj) return FHT_EUNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return FHT_EINVAL;
    std::vector<CallPtrs> calls(plan->count);
    for (int j = 0; j < plan->count; ++j) {
        const fht_adjoint_desc &dj = descs[j];
        if (!dj.grad_hough || !dj.grad_img || dj.grad_hough_pitch < plan->cols[j] ||
            dj.grad_img_pitch < plan->w[j])
            return FHT_EINVAL;
        calls[j] = CallPtrs{dj.grad_hough, dj.grad_hough_pitch, dj.grad_img, dj.grad_img_pitch};
    }
    const int mb = plan->minb;
    const Kernel k = plan->q == 0 ? kernel_adj_q0(mb) : plan->q == 1 ? kernel_adj_q1(mb)
                   : plan->q == 2 ? kernel_adj_q2(mb) : kernel_adj_q3(mb);
    return launch_table(plan, plan->adj, calls.data(), k, "batched_adjoint_f32", workspace,
                        stream);
}

fht_status fht_batched_status(const fht_plan *plan, const void *workspace, void *stream) {
    if (!plan || !workspace) return FHT_EINVAL;
    int err = 0;
    const unsigned char *ws = static_cast<const unsigned char *>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&err, ws + plan->last_counters_off + offsetof(Counters, error), sizeof(int),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FHT_ECUDA;
    return err == 0 ? FHT_OK : (fht_status)err;
}

fht_status fht_set_batched_tuning(const fht_batched_tuning *t) {
    const fht_batched_tuning v = t ? *t : default_batched_tuning();
    if (!batched_tuning_ok(v)) return FHT_EINVAL;
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune = v;
    return FHT_OK;
}

fht_status fht_get_batched_tuning(fht_batched_tuning *out) {
    if (!out) return FHT_EINVAL;
    std::lock_guard<std::mutex> lk(g_btune_mu);
    *out = g_btune;
    return FHT_OK;
}

fht_status fht_batched_test_hooks(fht_plan *plan, long long wait_budget_cycles, int dep_bias) {
    if (!plan || wait_budget_cycles <= 0 || dep_bias < 0) return FHT_EINVAL;
    plan->wait_budget = wait_budget_cycles;
    plan->dep_bias = dep_bias;
    return FHT_OK;
}

void fht_plan_destroy(fht_plan *plan) {
    if (!plan) return;
    release_table(plan->fwd);
    release_table(plan->adj);
    delete plan;
}

}  // extern "C"
