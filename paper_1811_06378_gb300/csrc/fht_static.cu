// fht_static.cu -- fht_forward_static: the single-quadrant forward transform
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc, or any routine that allocates: code
// running under an allocator or memory pool it does not own (a framework's
// caching allocator, a real-time path with a fixed memory budget), or a
// plugin host that forbids allocation after start-up. fht_forward needs scratch for its intermediate butterfly levels, which
// its caller must allocate. This entry point instead keeps that scratch in a
// fixed device array defined in this file: the library allocates nothing at
// call time, and every GPU that loads the library holds the array until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fht.h"

namespace {

// The fixed scratch: 64 MiB, enough for a uint8 -> int32 quadrant of a
// 4096 x 4096 image (its one intermediate level takes 34 MB as uint16).
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the array's device address, and the context it was looked up
// in. A context torn down and created again (cudaDeviceReset) loads the
// library's module afresh, at a new address, so the lookup is repeated when
// the current context is not the one recorded.
void *g_scratch_ptr[kMaxDevices] = {};
void *g_scratch_ctx[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, found through the runtime (the library links
// no driver library); nullptr if unavailable.
using CtxGetCurrent = int (*)(void **);
CtxGetCurrent ctx_get_current() {
    static CtxGetCurrent fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    return fn;
}

// Device address of the scratch on the current device. In host code the
// array's name is only a stand-in, so the address comes from
// cudaGetSymbolAddress, with that device current: once per device and
// context.
fht_status scratch_on_current_device(void **ptr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return FHT_ECUDA;
    void *ctx = nullptr;
    if (CtxGetCurrent f = ctx_get_current()) {
        if (f(&ctx) != 0) ctx = nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();   // do not leave this error for the caller's next check
            return FHT_ECUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *ptr = g_scratch_ptr[dev];
    return FHT_OK;
}

}  // namespace

extern "C" fht_status fht_forward_static(const void *img, fht_dtype in_t, int h, int w,
                                         int64_t in_pitch, fht_quadrant q, void *out,
                                         fht_dtype acc_t, int64_t out_pitch, void *stream) {
    size_t need = 0;
    fht_status s = fht_workspace_size(h, w, FHT_LAYOUT_QUADRANT, q, in_t, acc_t, &need);
    if (s != FHT_OK) return s;
    if (need > kStaticScratchBytes) return FHT_ENOMEM;   // beyond the fixed maximum
    void *scratch = nullptr;
    if (need > 0) {
        s = scratch_on_current_device(&scratch);
        if (s != FHT_OK) return s;
    }
    // Nothing in the scratch needs to start at zero: every intermediate
    // element the forward transform reads was written earlier in the same call.
    return fht_forward(img, in_t, h, w, in_pitch, q, out, acc_t, out_pitch, scratch,
                       need > 0 ? kStaticScratchBytes : 0, stream);
}
