// fht_host.h -- host-side declarations shared by the library's translation
// units: launch accounting and the per-type fused-pass launchers.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "fht_common.cuh"

namespace fht {

// Counts a kernel launch and, while profiling is on (fht_profile_begin),
// brackets it with CUDA events on its stream: construct right before the
// launch, call done() right after it. alg_bytes: the bytes the launch must
// move at least (the level it reads as stored plus the level it writes).
class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t st, double alg_bytes);
    void done();

  private:
    cudaStream_t st_;
    double bytes_;
    bool on_ = false;
    std::string name_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// Device-side wait-timeout counters (one per translation unit that holds
// pipelined kernels): each registers a function that returns its count and
// resets it; read_device_counters sums them. Registration returns true so it
// can initialise a namespace-scope constant.
bool register_device_counter(unsigned int (*read_and_reset)());
unsigned int read_device_counters();

// Whether two-block passes run as the persistent pipelined kernel
// (FHT_PIPE=1 in the environment turns it on; off by default).
bool pipe_enabled();

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

}  // namespace fht
