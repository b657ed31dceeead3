// Host-side helpers of libringo: status/error reporting, the device memory
// pool, pinned staging buffers and the optional per-kernel event timer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <string>

namespace ringo {

// Per-thread last error message (returned by ringo_last_error()).
void set_error(const std::string& msg);
const char* last_error();

// Stream-ordered allocation from a per-device pool that keeps freed memory
// cached for the next call.  Returns nullptr on failure (message recorded).
void* pool_alloc(size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);
// Free device memory plus the pool's cached, unused bytes.
uint64_t pool_available();
// Test hook: the spin bound armed for the next conversion (0: none); taking
// it disarms it.
uint32_t take_lookback_timeout();

// Pinned host staging buffers, cached and reused.
void* pinned_get(size_t bytes);
void pinned_put(void* p);

// Kernel timing with CUDA events (active between ringo_profile_start/stop).
bool profiling_enabled();
struct ProfScope {
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t start_ = nullptr;
};
// Host wall time of a scope, reported beside the kernels (name "host:...").
struct HostScope {
  explicit HostScope(const char* name);
  ~HostScope();
  const char* name_;
  std::chrono::steady_clock::time_point t0_;
  bool on_ = false;
};

}  // namespace ringo

#define RINGO_CUDA_TRY(expr)                                                        \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::ringo::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
      return (_e == cudaErrorMemoryAllocation) ? RINGO_ENOMEM : RINGO_ECUDA;        \
    }                                                                               \
  } while (0)

#define RINGO_LAUNCH_CHECK(name)                                                    \
  do {                                                                              \
    cudaError_t _e = cudaGetLastError();                                            \
    if (_e != cudaSuccess) {                                                        \
      ::ringo::set_error(std::string("launch of ") + (name) + ": " +                \
                         cudaGetErrorString(_e));                                   \
      return RINGO_ECUDA;                                                           \
    }                                                                               \
  } while (0)
