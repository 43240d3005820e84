// fht_debug.cuh -- bounds checks of the debug build (compiled with
// -DFHT_DEBUG: paper_1811_06378_gb300/build.py --debug, loaded by the package
// when FHT_DEBUG=1). The release build compiles none of this: every check
// below is the constant true there.
//
// The host records, in every pass descriptor, how many bytes from each
// side's pointer the pass may touch (PassDesc::dbg_lo_bytes / dbg_hi_bytes:
// the level buffer, or the caller's image / output view). Each CTA keeps
// those spans in shared memory; every global load or store of the pass
// kernels first checks that its elements lie inside them (a load may also
// read the destination: the image gradient an adjoint adds into). An access
// outside is skipped (a load gives zeros) and counted in a device word of
// the translation unit; fht_device_status reports FHT_EBOUNDS when any count
// is non-zero. A span of 0 bytes is not checked.
#pragma once

#include <cstdint>

#include "fht_common.cuh"

#ifdef FHT_DEBUG
#include "fht_host.h"
#endif

namespace fht {

#ifdef FHT_DEBUG

struct DebugSpan {
    uintptr_t lo, lo_end, hi, hi_end;
};

__device__ __forceinline__ DebugSpan *debug_span() {
    __shared__ DebugSpan s;
    return &s;
}

// Accesses refused in this translation unit since the host last read it.
static __device__ unsigned int g_fht_debug_refused = 0;

__device__ __forceinline__ bool debug_in(uintptr_t a, size_t n, uintptr_t b, uintptr_t e) {
    return a >= b && a + n <= e;
}

__device__ __forceinline__ bool debug_load_ok(const void *p, size_t n) {
    const DebugSpan &s = *debug_span();
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (s.lo_end == s.lo || debug_in(a, n, s.lo, s.lo_end) ||
        (s.hi_end != s.hi && debug_in(a, n, s.hi, s.hi_end)))
        return true;
    atomicAdd(&g_fht_debug_refused, 1u);
    return false;
}

__device__ __forceinline__ bool debug_store_ok(const void *p, size_t n) {
    const DebugSpan &s = *debug_span();
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (s.hi_end == s.hi || debug_in(a, n, s.hi, s.hi_end)) return true;
    atomicAdd(&g_fht_debug_refused, 1u);
    return false;
}

// Every thread of the CTA calls this before the pass's first access.
__device__ __forceinline__ void debug_begin(const PassDesc &d) {
    if (threadIdx.x == 0) {
        DebugSpan &s = *debug_span();
        s.lo = reinterpret_cast<uintptr_t>(d.lo.ptr);
        s.lo_end = s.lo + (uintptr_t)d.dbg_lo_bytes;
        s.hi = reinterpret_cast<uintptr_t>(d.hi.ptr);
        s.hi_end = s.hi + (uintptr_t)d.dbg_hi_bytes;
    }
    __syncthreads();
}

namespace {
unsigned int debug_read_and_reset() {
    unsigned int v = 0;
    const unsigned int zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_fht_debug_refused, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_fht_debug_refused, &zero, sizeof zero) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
const bool g_fht_debug_registered = register_device_counter(&debug_read_and_reset);
}  // namespace

#define FHT_LOAD_OK(p, n) (::fht::debug_load_ok((p), (n)))
#define FHT_STORE_OK(p, n) (::fht::debug_store_ok((p), (n)))
#define FHT_DEBUG_BEGIN(d) ::fht::debug_begin(d)

#else

#define FHT_LOAD_OK(p, n) (true)
#define FHT_STORE_OK(p, n) (true)
#define FHT_DEBUG_BEGIN(d) ((void)0)

#endif

}  // namespace fht
