// Small device-side building blocks: relaxed GPU-scope loads/stores, lane
// masks, block scans and the single-pass (decoupled look-back) tile prefix
// used by the compaction kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ringo_internal.cuh"

namespace ringo {

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
// Back off in a spin loop; true once the wait has exceeded kSpinLimit.
__device__ __forceinline__ bool spin_backoff(uint32_t& spins) {
  ++spins;
  if (spins > 32) __nanosleep(spins > 4096 ? 512 : 64);
  return spins > kSpinLimit;
}

// ---- mbarrier + bulk asynchronous copy (global -> shared) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from
// global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bounded wait for a bulk copy phase.  Gives up (returns false) after about a
// second, or at once when another block has already recorded an error.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  const volatile uint32_t* err) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if (err && (spins & 1023) == 0 && *err) return false;
    if (spins > kSpinLimit) return false;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// Exclusive sum over the block of one value per thread.  `sw` needs
// THREADS/32 + 1 entries.  Ends with __syncthreads(); `sw` may be reused after
// the caller's next barrier.
template <int THREADS, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* sw, T& total) {
  constexpr int NW = THREADS / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = warp_inclusive_sum(v);
  if (lane == 31) sw[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < NW ? sw[lane] : T(0);
    T s = warp_inclusive_sum(t);
    if (lane < NW) sw[lane] = s - t;
    if (lane == 31) sw[NW] = s;
  }
  __syncthreads();
  total = sw[NW];
  return sw[w] + x - v;
}

// Single-pass tile prefix (decoupled look-back, Merrill & Garland 2016) over a
// 64-bit packed status array.  Called by warp 0 of the tile's block; every
// lane returns the exclusive prefix of `agg` over tiles [0, tile).  Waits are
// bounded: on expiry the error bit is raised and the partial prefix is used
// (the host then reports RINGO_ETIMEOUT and discards the result).
__device__ __forceinline__ uint64_t warp_lookback(uint64_t* status, uint32_t tile,
                                                  uint64_t agg, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_relaxed_u64(status, kScanInc | agg);
    return 0;
  }
  if (lane == 0) st_relaxed_u64(status + tile, kScanAgg | agg);
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  uint32_t spins = 0;
  bool gave_up = false;
  while (true) {
    const int64_t idx = j - lane;
    uint64_t s = idx >= 0 ? ld_relaxed_u64(status + idx) : kScanInc;
    while (__any_sync(0xFFFFFFFFu, (s >> 62) == 0)) {
      if (spin_backoff(spins) || ((spins & 255) == 0 && *(volatile uint32_t*)err)) {
        gave_up = true;
        break;
      }
      if ((s >> 62) == 0) s = ld_relaxed_u64(status + idx);
    }
    if (gave_up) {
      if (lane == 0) atomicOr(err, kErrScan);
      if ((s >> 62) == 0) s = kScanInc;  // treat as zero-valued end
    }
    const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (s >> 62) == 2);
    const int first = inc ? __ffs(inc) - 1 : 32;
    uint64_t v = lane <= first ? (s & kScanValMask) : 0;
    excl += warp_sum(v);
    if (inc) break;
    j -= 32;
  }
  if (lane == 0) st_relaxed_u64(status + tile, kScanInc | (excl + agg));
  return excl;
}

}  // namespace ringo
