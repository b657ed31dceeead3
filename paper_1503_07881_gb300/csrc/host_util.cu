// Host-side helpers: error strings, device memory pool, pinned staging
// buffers and the per-kernel event timer.
#include "host_util.h"

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ringo.h"
#include "ringo_internal.cuh"

namespace ringo {

// ------------------------------------------------------------ errors ------
static thread_local std::string t_error;
void set_error(const std::string& msg) { t_error = msg; }
const char* last_error() { return t_error.c_str(); }

// ------------------------------------------------------------ pool --------
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t device_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = UINT64_MAX;  // keep freed memory for reuse by later calls
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  g_pools[dev] = pool;
  return pool;
}

// ------------------------------------------------------------ test hooks --
// Failures made on the host for the failure-detection tests: nothing on the
// device faults or hangs.  g_fail_countdown: allocations left to succeed
// before one fails (-1: none armed).  g_lookback_timeout: spin bound given
// to the next conversion, whose first radix pass then never claims its
// first tile, so that tile's successors wait on it until the bound.
static std::atomic<int64_t> g_fail_countdown{-1};
static std::atomic<uint32_t> g_lookback_timeout{0};

static bool injected_alloc_failure() {
  int64_t c = g_fail_countdown.load();
  while (c >= 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

uint32_t take_lookback_timeout() { return g_lookback_timeout.exchange(0u); }

void* pool_alloc(size_t bytes, cudaStream_t s) {
  if (injected_alloc_failure()) {
    set_error(std::string("device allocation of ") + std::to_string(bytes) +
              " bytes failed: injected failure (test hook)");
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return nullptr;
  }
  cudaMemPool_t pool = device_pool(dev);
  if (!pool) {
    set_error("cudaMemPoolCreate failed");
    return nullptr;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 256, pool, s);
  if (e != cudaSuccess) {
    // the pool keeps freed memory; give back what is unused and retry once
    cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(&p, bytes ? bytes : 256, pool, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("device allocation of ") + std::to_string(bytes) +
              " bytes failed: " + cudaGetErrorString(e));
    return nullptr;
  }
  return p;
}

void pool_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// Device bytes a new allocation can get: free device memory plus what the
// pool holds unused.
uint64_t pool_available() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  uint64_t held = 0, used = 0;
  cudaMemPool_t pool = device_pool(dev);
  if (pool) {
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &held);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  }
  return (uint64_t)free_b + (held > used ? held - used : 0);
}

// ------------------------------------------------------------ pinned ------
static std::mutex g_pin_mu;
static std::multimap<size_t, void*> g_pin_free;
static std::map<void*, size_t> g_pin_size;

void* pinned_get(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  auto it = g_pin_free.lower_bound(bytes);
  if (it != g_pin_free.end()) {
    void* p = it->second;
    g_pin_free.erase(it);
    return p;
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_pin_size[p] = bytes;
  return p;
}

void pinned_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace(g_pin_size[p], p);
}

// ------------------------------------------------------------ profiling ---
struct ProfRecord {
  std::string name;
  cudaEvent_t a, b;   // device interval (null for host records)
  double host_ms;     // host interval
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRecord> g_prof;
static std::vector<cudaEvent_t> g_event_cache;

static cudaEvent_t get_event() {
  if (!g_event_cache.empty()) {
    cudaEvent_t e = g_event_cache.back();
    g_event_cache.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool profiling_enabled() { return g_prof_on; }

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s_, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // kernels recorded into a graph are timed around the graph launch
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  start_ = get_event();
  cudaEventRecord(start_, s_);
}

ProfScope::~ProfScope() {
  if (!start_) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t end = get_event();
  cudaEventRecord(end, s_);
  g_prof.push_back(ProfRecord{name_, start_, end, 0.0});
}

HostScope::HostScope(const char* name) : name_(name) {
  if (g_prof_on) t0_ = std::chrono::steady_clock::now(), on_ = true;
}

HostScope::~HostScope() {
  if (!on_) return;
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back(ProfRecord{name_, nullptr, nullptr, ms});
}

}  // namespace ringo

extern "C" int ringo_profile_start(void) {
  std::lock_guard<std::mutex> lk(ringo::g_prof_mu);
  for (auto& r : ringo::g_prof) {
    if (!r.a) continue;
    ringo::g_event_cache.push_back(r.a);
    ringo::g_event_cache.push_back(r.b);
  }
  ringo::g_prof.clear();
  ringo::g_prof_on = true;
  return RINGO_OK;
}

extern "C" int ringo_profile_stop(ringo_kernel_stat* out, int32_t cap, int32_t* n_out) {
  std::lock_guard<std::mutex> lk(ringo::g_prof_mu);
  ringo::g_prof_on = false;
  std::vector<std::string> order;
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (auto& r : ringo::g_prof) {
    float ms = (float)r.host_ms;
    if (r.a && (cudaEventSynchronize(r.b) != cudaSuccess ||
                cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)) {
      ringo::set_error("profiling event failed");
      return RINGO_ECUDA;
    }
    if (!agg.count(r.name)) order.push_back(r.name);
    auto& a = agg[r.name];
    a.first += 1;
    a.second += ms;
  }
  int32_t n = 0;
  for (auto& name : order) {
    if (out && n < cap) {
      memset(&out[n], 0, sizeof(out[n]));
      strncpy(out[n].name, name.c_str(), sizeof(out[n].name) - 1);
      out[n].launches = agg[name].first;
      out[n].total_ms = agg[name].second;
    }
    ++n;
  }
  if (n_out) *n_out = n;
  for (auto& r : ringo::g_prof) {
    if (!r.a) continue;
    ringo::g_event_cache.push_back(r.a);
    ringo::g_event_cache.push_back(r.b);
  }
  ringo::g_prof.clear();
  return RINGO_OK;
}

extern "C" int ringo_test_inject_alloc_failure(int32_t skip) {
  ringo::g_fail_countdown.store(skip < 0 ? -1 : (int64_t)skip);
  return RINGO_OK;
}

extern "C" int ringo_test_inject_lookback_timeout(uint32_t spin_limit) {
  if (spin_limit == 0 || spin_limit > ringo::kSpinLimit) {
    ringo::set_error("ringo_test_inject_lookback_timeout: spin_limit outside [1, 2^21]");
    return RINGO_EINVAL;
  }
  ringo::g_lookback_timeout.store(spin_limit);
  return RINGO_OK;
}

extern "C" int ringo_test_pool_used(uint64_t* bytes) {
  if (!bytes) return RINGO_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    ringo::set_error("no usable current device");
    return RINGO_ECUDA;
  }
  cudaMemPool_t pool = ringo::device_pool(dev);
  if (!pool) return RINGO_ECUDA;
  uint64_t used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return RINGO_ECUDA;
  }
  *bytes = used;
  return RINGO_OK;
}
