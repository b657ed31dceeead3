// Small device-side building blocks: relaxed GPU-scope loads/stores, lane
// masks, block scans, bulk asynchronous copies, and the single-pass
// (decoupled look-back, Merrill & Garland 2016) tile prefix used by the
// compaction kernels, here in a two-level form (tiles within a chunk, then
// chunk aggregates).
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
// Back off in a spin loop; true once the wait has exceeded `limit` spins
// (0: kSpinLimit).
__device__ __forceinline__ bool spin_backoff(uint32_t& spins, uint32_t limit = 0) {
  ++spins;
  if (spins > 32) __nanosleep(spins > 4096 ? 512 : 64);
  return spins > (limit ? limit : kSpinLimit);
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Barrier among the first `count` threads of the block (named barrier `id`;
// 0 is the one __syncthreads uses).
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
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
// Asks the memory system to bring `bytes` (multiple of 16; 16-byte aligned
// address) from global memory into L2, with no destination in this block.
__device__ __forceinline__ void bulk_prefetch_l2(const void* gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}
// Bounded wait for a bulk copy phase.  Gives up (returns false) after about a
// second, or at once when another block has already recorded an error.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  const volatile uint32_t* err,
                                                  uint32_t limit = 0) {
  const uint32_t lim = limit ? limit : kSpinLimit;
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if (err && (spins & 1023) == 0 && *err) return false;
    if (spins > lim) return false;
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
// Largest r in [0, V) with off[r] <= e, for a non-decreasing off with
// off[0] <= e < off[V], found by one warp (all lanes call it): each round
// splits [lo, hi) into 32 parts and the lanes test the part starts together,
// so the search takes log32(V) dependent loads instead of log2(V).
__device__ __forceinline__ uint32_t warp_owner(const int64_t* __restrict__ off, uint32_t V, uint64_t e,
                                               int lane) {
  uint32_t lo = 0, hi = V;  // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) >> 5;
    const uint32_t c = lo + (uint32_t)lane * step;
    const bool le = lane > 0 && c < hi && (uint64_t)off[c] <= e;
    // off is non-decreasing, so the lanes that pass are 1 .. k
    const uint32_t k = __popc(__ballot_sync(0xFFFFFFFFu, le));
    const uint32_t nhi = lo + (k + 1) * step;
    lo += k * step;
    hi = nhi < hi ? nhi : hi;
  }
  return lo;
}

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

// Chunk arrays of the two-level single-value look-back (one set per scan).
struct ScanChunks {
  uint64_t* agg;   // [chunks] packed sums added by the chunk's tiles
  uint64_t* inc;   // [chunks] kScanInc | inclusive prefix once known
  uint32_t* cnt;   // [chunks] tiles that have added their value
  uint32_t limit;  // bound of the waits (0: kSpinLimit)
  // 1: every chunk's two sums stay below 2^24 (a chunk covers at most 2^17
  // items), so agg holds (tiles added << 48) | (A << 24) | B in one word: a
  // single relaxed load says whether the chunk is complete, no counter or
  // fence is needed.  0: agg holds the packed sums and cnt counts the tiles.
  uint32_t small;
};

__device__ __forceinline__ uint64_t chunk_word(uint64_t agg) {
  return (1ull << 48) | ((uint64_t)unpackA(agg) << 24) | (uint64_t)unpackB(agg);
}
__device__ __forceinline__ uint64_t chunk_sums(uint64_t w) {
  return pack2((uint32_t)(w >> 24) & 0xFFFFFFu, (uint32_t)w & 0xFFFFFFu);
}

// Two-level tile prefix for the compaction kernels: like warp_lookback, but a
// tile walks back only within its kChunkTiles-tile chunk and then over chunk
// aggregates (complete once every tile of the chunk has added its value), so
// no tile waits on the chain of inclusive prefixes of all its predecessors.
// Called by warp 0 of the block; all lanes return the exclusive prefix.
__device__ __forceinline__ uint64_t warp_lookback2(uint64_t* status, ScanChunks ch, uint32_t tile,
                                                   uint32_t ntiles, uint64_t agg, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const uint32_t c = tile >> kChunkShift;
  const uint32_t first = c << kChunkShift;
  // publish this tile's value, and add it to the chunk aggregate
  if (lane == 0) {
    st_relaxed_u64(status + tile, (tile == 0 ? kScanInc : kScanAgg) | agg);
    if (ch.small) {
      atomicAdd((unsigned long long*)(ch.agg + c), (unsigned long long)chunk_word(agg));
    } else {
      if (agg) atomicAdd((unsigned long long*)(ch.agg + c), (unsigned long long)agg);
      __threadfence();
      atomicAdd(ch.cnt + c, 1u);
    }
  }
  uint64_t excl = 0;
  if (tile == 0) return 0;
  uint32_t spins = 0;
  const volatile uint32_t* verr = err;
  // 1. earlier tiles of this chunk (at most 31: one warp-wide read).  Lane l
  //    reads tile - 1 - l; the nearest inclusive prefix ends the sum, and
  //    every tile before it (in lane order) must have published.
  const int cnt_in = (int)(tile - first);
  if (cnt_in > 0) {
    while (true) {
      const bool in_chunk = lane < cnt_in;
      const uint64_t s = in_chunk ? ld_relaxed_u64(status + (tile - 1 - lane)) : 0;
      const uint32_t incm = __ballot_sync(0xFFFFFFFFu, in_chunk && (s >> 62) == 2);
      const int stop = incm ? __ffs(incm) - 1 : cnt_in;
      const uint32_t missing = __ballot_sync(0xFFFFFFFFu, lane < stop && (s >> 62) == 0);
      if (missing) {
        if (spin_backoff(spins, ch.limit) || ((spins & 255) == 0 && *verr)) {
          if (lane == 0) atomicOr(err, kErrScan);
          return excl;
        }
        continue;
      }
      const uint64_t v = (lane < stop || (incm && lane == stop)) ? (s & kScanValMask) : 0;
      excl = warp_sum(v);
      if (incm) return excl;
      break;
    }
  }
  // 2. earlier chunks, 32 per round
  int64_t cc = (int64_t)c - 1;
  while (cc >= 0) {
    const int64_t k = cc - lane;
    uint64_t inc = 0, word = 0;
    uint32_t done = 0;
    if (k >= 0) {
      inc = ld_relaxed_u64(ch.inc + k);
      const uint32_t need = min((uint32_t)kChunkTiles, ntiles - ((uint32_t)k << kChunkShift));
      if (ch.small) {
        word = ld_relaxed_u64(ch.agg + k);
        done = (uint32_t)(word >> 48) >= need ? 1u : 0u;
      } else {
        done = ld_acquire_u32(ch.cnt + k) >= need ? 1u : 0u;
      }
    }
    const uint32_t incm = __ballot_sync(0xFFFFFFFFu, k >= 0 && (inc >> 62) == 2);
    const int stop = incm ? __ffs(incm) - 1 : 32;
    const uint32_t ready = __ballot_sync(0xFFFFFFFFu, k < 0 || done || lane >= stop);
    if (ready != 0xFFFFFFFFu) {
      if (spin_backoff(spins, ch.limit) || ((spins & 255) == 0 && *verr)) {
        if (lane == 0) atomicOr(err, kErrScan);
        return excl;
      }
      continue;
    }
    uint64_t v = 0;
    if (k >= 0 && lane < stop) v = ch.small ? chunk_sums(word) : ld_relaxed_u64(ch.agg + k);
    if (lane == stop) v = inc & kScanValMask;
    excl += warp_sum(v);
    if (incm) return excl;
    cc -= 32;
  }
  return excl;
}

// After its look-back the first tile of a chunk knows the previous chunk's
// inclusive prefix, and the last tile knows its own chunk's.
__device__ __forceinline__ void publish_chunk_inc(ScanChunks ch, uint32_t tile, uint32_t ntiles,
                                                  uint64_t excl, uint64_t agg) {
  const uint32_t c = tile >> kChunkShift;
  if ((tile & (kChunkTiles - 1)) == 0 && c > 0) st_relaxed_u64(ch.inc + c - 1, kScanInc | excl);
  if ((tile & (kChunkTiles - 1)) == kChunkTiles - 1 || tile == ntiles - 1)
    st_relaxed_u64(ch.inc + c, kScanInc | (excl + agg));
}

// Exclusive prefix of `agg` over earlier tiles (two-level look-back) and the
// publication of this tile's (and, where it knows one, a chunk's) inclusive
// prefix.  Warp 0 only; every lane returns the prefix.
__device__ __forceinline__ uint64_t scan_prefix(uint64_t* status, ScanChunks ch, uint32_t tile,
                                                uint32_t ntiles, uint64_t agg, uint32_t* err) {
  const uint64_t excl = warp_lookback2(status, ch, tile, ntiles, agg, err);
  if ((threadIdx.x & 31) == 0) {
    st_relaxed_u64(status + tile, kScanInc | (excl + agg));
    publish_chunk_inc(ch, tile, ntiles, excl, agg);
  }
  return excl;
}

// Largest s with m.start[s] <= g (binary search over the segment starts).
__device__ __forceinline__ uint32_t seg_of(SegMap m, uint32_t g) {
  uint32_t lo = 0, hi = m.nseg;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(m.start + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Thread 0 claims the next global slot and resolves it; the result is
// shared through `out` (shared memory) after the caller's barrier.
struct Claim {
  uint32_t seg;
  uint32_t tile;   // local tile of the segment
  uint32_t valid;  // 0: past the last slot
  uint32_t slot;   // the global slot
};
__device__ __forceinline__ Claim claim_next(SegMap m, uint32_t* counter) {
  Claim c;
  const uint32_t g = atomicAdd(counter, 1u);
  c.slot = g;
  if (g >= __ldg(m.start + m.nseg)) {
    c.seg = 0;
    c.tile = 0;
    c.valid = 0;
    return c;
  }
  // one segment (a single table): its slots start at 0, nothing to search
  c.seg = m.nseg > 1 ? seg_of(m, g) : 0u;
  c.tile = m.nseg > 1 ? g - __ldg(m.start + c.seg) : g;
  c.valid = 1;
  return c;
}
__device__ __forceinline__ void claim_slot(SegMap m, uint32_t* counter, Claim* out) {
  const uint32_t g = atomicAdd(counter, 1u);
  out->slot = g;
  if (g >= __ldg(m.start + m.nseg)) {
    out->valid = 0;
    return;
  }
  // one segment (a single table): its slots start at 0, nothing to search
  const uint32_t sidx = m.nseg > 1 ? seg_of(m, g) : 0u;
  out->seg = sidx;
  out->tile = m.nseg > 1 ? g - __ldg(m.start + sidx) : g;
  out->valid = 1;
}

}  // namespace ringo
