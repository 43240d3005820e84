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
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fht.h"
#include "fht_batched.cuh"
#include "fht_host.h"

using namespace fht;
using namespace fht::batched;

// Direct launches of one plan stage their segment tables in turn in this
// many pinned tables, so the host can run that many launches ahead.
constexpr int kDirectTables = 3;

struct fht_plan {
    int count = 0;
    int f32 = 0;
    int sigma = 1;
    int n_segs = 0, total_items = 0;
    size_t table_bytes = 0, counters_off = 0, done_off = 0, levels_off = 0;
    size_t ws_bytes = 0, smem = 0;
    int n_done = 0;
    std::vector<int> h, w, rows, cols;   // per image: size, and its quadrant's n x W
    // pinned staging of the segment table: kDirectTables tables used in turn
    // by direct launches (each reused only once its previous copy has run),
    // then one for the latest stream capture
    void *host_table = nullptr;
    cudaEvent_t copied[kDirectTables] = {};   // after each direct table's last copy
    bool copy_pending[kDirectTables] = {};
    int next_table = 0;
    long long wait_budget = 4000000000LL;   // ~2 s of SM clocks
    int dep_bias = 0;
};

namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

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
    std::vector<BatchSeg> segs;
    std::vector<size_t> level_off;
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
        const int transpose = q >= 2, sigma = (q == 0 || q == 3) ? 1 : -1;
        const int h_c = transpose ? ws[j] : hs[j], w_c = transpose ? hs[j] : ws[j];
        const int n = rows, W = cols;
        int ms[2], npass;
        if (K <= 6) {
            ms[0] = K;
            npass = 1;
        } else {
            ms[0] = (K + 1) / 2;
            ms[1] = K / 2;
            npass = 2;
        }
        // the one intermediate level (after pass 0), uint16 for uint8 images
        size_t lvl_off = 0;
        int lvl_cols = 0;
        int64_t lvl_pitch = 0;
        const int lvl_type = f32 ? kF32 : kU16;
        if (npass == 2) {
            lvl_cols = std::min(W, w_c + (1 << ms[0]));
            lvl_pitch = (lvl_cols + 63) / 64 * 64;
            lvl_off = level_bytes;
            level_bytes += align256((size_t)n * lvl_pitch * (f32 ? 4 : 2));
        }
        int prev_items = 0;
        for (int p = 0; p < npass; ++p) {
            const int m = ms[p], k0 = p == 0 ? 0 : ms[0], k1 = k0 + m;
            BatchSeg s{};
            PassDesc &d = s.d;
            d.lo_image = p == 0;
            d.transpose = transpose;
            d.hi_final = p == npass - 1;
            d.n = n;
            d.W = W;
            d.K = K;
            d.k0 = k0;
            d.sigma = sigma;
            d.a_lo = 0;
            d.a_count = 1 << k0;
            d.need_lo = 0;
            d.need_hi = (1 << k1) - 1;
            d.s_count = n >> k1;
            d.t_first = 0;
            d.t_last = n - 1;
            d.row_base = 0;
            d.row_dir = 1;
            d.shift_win = w_c;
            d.black_wc = w_c;
            d.lo = p == 0 ? Side{nullptr, 0, f32 ? kF32 : kU8, h_c, w_c}
                          : Side{nullptr, lvl_pitch, lvl_type, n, lvl_cols};
            d.hi = d.hi_final ? Side{nullptr, 0, f32 ? kF32 : kI32, 0, W}
                              : Side{nullptr, lvl_pitch, lvl_type, n, lvl_cols};
            d.p_begin = 0;
            d.p_count = d.hi.cols;
            const bool u16_mid = u8 && p == 0;
            if (m >= 4) {
                const int rb = 1 << (m - 3);
                d.n_a = std::max(u16_mid ? 2 : 1, 8 / rb);
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
            s.chunk = std::max(1, std::min(kUnitsPerItem, s.units));
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
    fht_plan *P = new (std::nothrow) fht_plan();
    if (!P) return FHT_ENOMEM;
    P->count = count;
    P->f32 = f32;
    P->sigma = (q == 0 || q == 3) ? 1 : -1;
    P->n_segs = (int)segs.size();
    P->total_items = items;
    P->n_done = n_done;
    P->smem = smem;
    P->table_bytes = segs.size() * sizeof(BatchSeg);
    P->counters_off = align256(P->table_bytes);
    P->done_off = P->counters_off + 256;
    P->levels_off = align256(P->done_off + (size_t)n_done * sizeof(unsigned int));
    // intermediate offsets inside the workspace
    for (auto &s : segs) {
        s.lo_off += (int64_t)P->levels_off;
        s.hi_off += (int64_t)P->levels_off;
    }
    P->ws_bytes = P->levels_off + level_bytes;
    for (int j = 0; j < count; ++j) {
        int r = 0, c = 0;
        fht_query_shape(hs[j], ws[j], q, &r, &c);
        P->h.push_back(hs[j]);
        P->w.push_back(ws[j]);
        P->rows.push_back(r);
        P->cols.push_back(c);
    }
    if (cudaMallocHost(&P->host_table, (kDirectTables + 1) * P->counters_off) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return FHT_ENOMEM;
    }
    for (int c = 0; c < kDirectTables; ++c) {
        if (cudaEventCreateWithFlags(&P->copied[c], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            fht_plan_destroy(P);
            return FHT_ECUDA;
        }
    }
    for (int c = 0; c <= kDirectTables; ++c)
        std::memcpy(static_cast<unsigned char *>(P->host_table) + c * P->counters_off,
                    segs.data(), P->table_bytes);
    *plan = P;
    *workspace_bytes = P->ws_bytes;
    return FHT_OK;
}

fht_status fht_forward_batched(fht_plan *plan, const fht_image_desc *descs, void *workspace,
                               size_t workspace_bytes, void *stream) {
    if (!plan || !descs || !workspace || workspace_bytes < plan->ws_bytes) return FHT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return FHT_EINVAL;
    for (int j = 0; j < plan->count; ++j) {
        const fht_image_desc &dj = descs[j];
        if (!dj.img || !dj.out || dj.img_pitch < plan->w[j] || dj.out_pitch < plan->cols[j])
            return FHT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FHT_ECUDA;
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    // a direct launch takes the next table of the ring, once the copy of the
    // launch that used it last has read it
    const int tab = capturing ? kDirectTables : plan->next_table;
    if (!capturing) {
        plan->next_table = (plan->next_table + 1) % kDirectTables;
        if (plan->copy_pending[tab]) {
            if (cudaEventSynchronize(plan->copied[tab]) != cudaSuccess) return FHT_ECUDA;
            plan->copy_pending[tab] = false;
        }
    }
    unsigned char *table = static_cast<unsigned char *>(plan->host_table) +
                           (size_t)tab * plan->counters_off;
    BatchSeg *segs = reinterpret_cast<BatchSeg *>(table);
    for (int i = 0; i < plan->n_segs; ++i) {
        BatchSeg &sg = segs[i];
        const fht_image_desc &im = descs[sg.image];
        if (sg.lo_from_image) {
            sg.d.lo.ptr = const_cast<void *>(im.img);
            sg.d.lo.pitch = im.img_pitch;
        } else {
            sg.d.lo.ptr = ws + sg.lo_off;
        }
        if (sg.hi_from_image) {
            sg.d.hi.ptr = im.out;
            sg.d.hi.pitch = im.out_pitch;
        } else {
            sg.d.hi.ptr = ws + sg.hi_off;
        }
    }
    cudaError_t e = cudaMemcpyAsync(ws, table, plan->counters_off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !capturing) {
        e = cudaEventRecord(plan->copied[tab], st);
        if (e == cudaSuccess) plan->copy_pending[tab] = true;
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ws + plan->counters_off, 0,
                            plan->levels_off - plan->counters_off, st);
    if (e != cudaSuccess) return FHT_ECUDA;
    const Kernel k = plan->f32 ? (plan->sigma > 0 ? kernel_f32_pos() : kernel_f32_neg())
                               : (plan->sigma > 0 ? kernel_u8_pos() : kernel_u8_neg());
    if (plan->smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem);
        if (e != cudaSuccess) return FHT_ECUDA;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, plan->smem);
    int grid = std::max(1, sms * std::max(per_sm, 1));
    grid = std::min(grid, std::max(plan->total_items, 1));
    LaunchScope scope(plan->f32 ? "batched_forward_f32" : "batched_forward_u8_i32", st, 0.0);
    k<<<grid, kWarps * 32, plan->smem, st>>>(
        reinterpret_cast<const BatchSeg *>(ws), plan->n_segs, plan->total_items,
        reinterpret_cast<Counters *>(ws + plan->counters_off),
        reinterpret_cast<unsigned int *>(ws + plan->done_off), plan->wait_budget,
        plan->dep_bias);
    scope.done();
    e = cudaGetLastError();
    return e == cudaSuccess ? FHT_OK : FHT_ECUDA;
}

fht_status fht_batched_status(const fht_plan *plan, const void *workspace, void *stream) {
    if (!plan || !workspace) return FHT_EINVAL;
    int err = 0;
    const unsigned char *ws = static_cast<const unsigned char *>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&err, ws + plan->counters_off + offsetof(Counters, error), sizeof(int),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FHT_ECUDA;
    return err == 0 ? FHT_OK : (fht_status)err;
}

fht_status fht_batched_test_hooks(fht_plan *plan, long long wait_budget_cycles, int dep_bias) {
    if (!plan || wait_budget_cycles <= 0 || dep_bias < 0) return FHT_EINVAL;
    plan->wait_budget = wait_budget_cycles;
    plan->dep_bias = dep_bias;
    return FHT_OK;
}

void fht_plan_destroy(fht_plan *plan) {
    if (!plan) return;
    for (int c = 0; c < kDirectTables; ++c) {
        if (!plan->copied[c]) continue;
        if (plan->copy_pending[c]) cudaEventSynchronize(plan->copied[c]);
        cudaEventDestroy(plan->copied[c]);
    }
    if (plan->host_table) cudaFreeHost(plan->host_table);
    delete plan;
}

}  // extern "C"
