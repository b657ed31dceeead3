// Select and join on edge tables (ringo_table_select, ringo_table_join): the
// relational operations that feed the conversion (Section 3.3, "Tables in
// Ringo"; Section 4, Table "table_ringo": select by comparison with a
// constant, in place; join with a single-column table, into a new table).
//
// Both are single-pass stable compactions over 4096-row tiles: a block loads
// its rows (each warp 512 consecutive rows, 32 per coalesced step), decides
// how many output rows each gives (0/1 for select; the key's multiplicity in
// the second table for join), and finds the tile's output offset with the two-level decoupled
// look-back over tiles claimed in order.  Select writes in place: a kept row
// moves to a position at or before its own, and a tile publishes its count
// only after it has loaded all its rows, so no row is overwritten before it
// is read.  Join first builds the set of the second table's keys with their
// multiplicities (an open-addressing hash table when that is small, else a
// bitmap over the key range with a hash table for the keys that occur more
// than once); a marking pass then records, per row, whether its key occurs
// once or more often (two bits per row) and scans the tiles' output counts,
// so the output size is known before anything is written; a writing pass
// copies the matching rows, skipping tiles without any.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kOpThreads = 256;
constexpr uint32_t kOpItems = 16;
constexpr uint32_t kOpTile = kOpThreads * kOpItems;  // 4096 rows
// a join's key hash table up to this size stays in cache; above it, a bitmap
// over the key range is used when that is smaller
constexpr uint64_t kJoinHashCacheBytes = 8ull << 20;
// a join's key hash table up to this many slots is copied into shared memory
constexpr uint32_t kJoinSmemSlots = 2048;

struct OpScan {
  uint64_t* status;  // [tiles]
  ScanChunks ch;     // chunk sums of the two-level look-back
  uint32_t* err;
  uint32_t* counter;  // tile claims
};

__device__ __forceinline__ bool compare(int32_t x, int op, int32_t v) {
  switch (op) {
    case RINGO_CMP_LT: return x < v;
    case RINGO_CMP_LE: return x <= v;
    case RINGO_CMP_EQ: return x == v;
    case RINGO_CMP_NE: return x != v;
    case RINGO_CMP_GE: return x >= v;
    default: return x > v;
  }
}

__device__ __forceinline__ uint32_t hash_slot(int32_t k, uint32_t mask) {
  return (uint32_t)(((uint64_t)(uint32_t)k * 0x9E3779B97F4A7C15ull) >> 32) & mask;
}

// multiplicity of k in the hash table (0 if absent)
__device__ __forceinline__ uint32_t lookup(const unsigned long long* table, uint32_t mask, int32_t k) {
  uint32_t h = hash_slot(k, mask);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long slot = table[h];
    if ((uint32_t)slot == 0u) return 0;
    if ((uint32_t)(slot >> 32) == (uint32_t)k) return (uint32_t)slot;
    h = (h + 1) & mask;
  }
  return 0;
}

__global__ void k_hash_build(const int32_t* __restrict__ keys, uint32_t nkeys,
                             unsigned long long* __restrict__ table, uint32_t mask) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x) {
    const int32_t k = keys[i];
    const unsigned long long mine = ((unsigned long long)(uint32_t)k << 32) | 1ull;
    uint32_t h = hash_slot(k, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      unsigned long long slot = table[h];
      if ((uint32_t)slot == 0u) {
        slot = atomicCAS(table + h, 0ull, mine);
        if (slot == 0ull) break;  // inserted
      }
      if ((uint32_t)(slot >> 32) == (uint32_t)k) {
        atomicAdd(table + h, 1ull);  // one more occurrence (count in the low half)
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

// The second table's keys: multiplicity of a key, 0 if absent.  Either an
// open-addressing hash table of (key, count) slots (bits == nullptr), or a
// bitmap over [kmin, kmin + range) of the keys present, a bitmap of those
// present more than once (dup, nullptr if none is) and a hash table of the
// latter's counts.
struct KeySet {
  const unsigned long long* table;
  uint32_t mask;
  const uint32_t* bits;
  const uint32_t* dup;
  int64_t kmin;
  uint64_t range;
};

__device__ __forceinline__ uint32_t multiplicity(const KeySet& ks, int32_t k) {
  if (!ks.bits) return lookup(ks.table, ks.mask, k);
  const uint64_t off = (uint64_t)((int64_t)k - ks.kmin);  // below kmin wraps past range
  if (off >= ks.range) return 0u;
  const uint32_t w = (uint32_t)(off >> 5), b = 1u << (off & 31);
  if (!(__ldg(ks.bits + w) & b)) return 0u;
  if (!ks.dup || !(__ldg(ks.dup + w) & b)) return 1u;
  return lookup(ks.table, ks.mask, k);
}

// mm[0] = min, mm[1] = max of the keys (mm preset to INT32_MAX, INT32_MIN)
__global__ void k_key_range(const int32_t* __restrict__ keys, uint32_t nkeys, int* __restrict__ mm) {
  int lo = 0x7FFFFFFF, hi = (int)0x80000000;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x) {
    lo = min(lo, keys[i]);
    hi = max(hi, keys[i]);
  }
  lo = __reduce_min_sync(0xFFFFFFFFu, lo);
  hi = __reduce_max_sync(0xFFFFFFFFu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(mm, lo);
    atomicMax(mm + 1, hi);
  }
}

// bits: every key; dup: keys met again; extra: the number of repeats
__global__ void k_bits_build(const int32_t* __restrict__ keys, uint32_t nkeys, int64_t kmin,
                             uint32_t* __restrict__ bits, uint32_t* __restrict__ dup,
                             unsigned long long* __restrict__ extra) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x) {
    const uint64_t off = (uint64_t)((int64_t)keys[i] - kmin);
    const uint32_t w = (uint32_t)(off >> 5), b = 1u << (off & 31);
    if (atomicOr(bits + w, b) & b) {
      atomicOr(dup + w, b);
      atomicAdd(extra, 1ull);
    }
  }
}

// (key, count) of every key that occurs more than once
__global__ void k_hash_dup(const int32_t* __restrict__ keys, uint32_t nkeys, int64_t kmin,
                           const uint32_t* __restrict__ dup, unsigned long long* __restrict__ table,
                           uint32_t mask) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x) {
    const int32_t k = keys[i];
    const uint64_t off = (uint64_t)((int64_t)k - kmin);
    if (!(dup[off >> 5] & (1u << (off & 31)))) continue;
    const unsigned long long mine = ((unsigned long long)(uint32_t)k << 32) | 1ull;
    uint32_t h = hash_slot(k, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      unsigned long long slot = table[h];
      if ((uint32_t)slot == 0u) {
        slot = atomicCAS(table + h, 0ull, mine);
        if (slot == 0ull) break;
      }
      if ((uint32_t)(slot >> 32) == (uint32_t)k) {
        atomicAdd(table + h, 1ull);
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

// Key-set forms of the join's marking pass.
enum JoinMode { kJoinSmemHash = 0, kJoinBitmap = 1, kJoinHash = 2 };

// 16-bit filter index of a key (multiplicative hashing, top bits)
__device__ __forceinline__ uint32_t filter_bit(int32_t k) { return ((uint32_t)k * 0x9E3779B1u) >> 16; }

// Join, marking pass: persistent blocks take 4096-row tiles in a fixed
// stride (no tile waits on another); warp w reads rows [tile * 4096 + 512 w,
// + 512), 32 per step.  flags[(tile * 8 + w) * 16 + step] = (rows whose key
// occurs, rows whose key occurs more than once) as lane bitmasks;
// tile_cnt[tile] = the tile's output rows.
//   kJoinSmemHash: a hash table of at most kJoinSmemSlots slots, copied into
//     shared memory with a 64K-bit filter of its keys; most absent keys cost
//     one filter test;
//   kJoinBitmap / kJoinHash: the key set in global memory, the first access
//     of all 16 rows of a thread issued before any is used.
template <int kMode>
__global__ void __launch_bounds__(kOpThreads)
    k_join_mark(const int32_t* __restrict__ keycol, uint32_t n, KeySet ks, uint2* __restrict__ flags,
                uint64_t* __restrict__ tile_cnt) {
  constexpr int kWarps = kOpThreads / 32;
  constexpr bool kSmem = kMode == kJoinSmemHash;
  __shared__ unsigned long long s_tab[kSmem ? kJoinSmemSlots : 1];
  __shared__ uint32_t s_filter[kSmem ? 2048 : 1];
  __shared__ unsigned long long s_w[2][kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (kSmem) {
    for (uint32_t i = tid; i < 2048; i += kOpThreads) s_filter[i] = 0;
    __syncthreads();
    for (uint32_t i = tid; i <= ks.mask; i += kOpThreads) {
      const unsigned long long v = ks.table[i];
      s_tab[i] = v;
      if ((uint32_t)v) {
        const uint32_t f = filter_bit((int32_t)(v >> 32));
        atomicOr(&s_filter[f >> 5], 1u << (f & 31));
      }
    }
    __syncthreads();
  }
  const uint32_t ntiles = (n + kOpTile - 1) / kOpTile;
  int buf = 0;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const uint32_t base = tile * kOpTile + (uint32_t)warp * (32 * kOpItems) + (uint32_t)lane;
    int32_t k[kOpItems];
#pragma unroll
    for (int q = 0; q < kOpItems; ++q) {
      const uint32_t r = base + 32u * q;
      k[q] = r < n ? keycol[r] : 0;
    }
    uint32_t m[kOpItems];
    if constexpr (kMode == kJoinSmemHash) {
#pragma unroll
      for (int q = 0; q < kOpItems; ++q) {
        const uint32_t f = filter_bit(k[q]);
        m[q] = 0u;
        if (base + 32u * q < n && ((s_filter[f >> 5] >> (f & 31)) & 1u)) m[q] = lookup(s_tab, ks.mask, k[q]);
      }
    } else if constexpr (kMode == kJoinBitmap) {
#pragma unroll
      for (int q = 0; q < kOpItems; ++q) {
        const uint64_t off = (uint64_t)((int64_t)k[q] - ks.kmin);
        m[q] = base + 32u * q < n && off < ks.range ? __ldg(ks.bits + (off >> 5)) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kOpItems; ++q) {
        const uint64_t off = (uint64_t)((int64_t)k[q] - ks.kmin);
        m[q] = (m[q] >> (off & 31)) & 1u;
        if (m[q] && ks.dup && ((__ldg(ks.dup + (off >> 5)) >> (off & 31)) & 1u))
          m[q] = lookup(ks.table, ks.mask, k[q]);
      }
    } else {
      unsigned long long sl[kOpItems];
#pragma unroll
      for (int q = 0; q < kOpItems; ++q)
        sl[q] = base + 32u * q < n ? ks.table[hash_slot(k[q], ks.mask)] : 0ull;
#pragma unroll
      for (int q = 0; q < kOpItems; ++q) {
        if ((uint32_t)sl[q] == 0u) m[q] = 0u;  // empty first slot (or past the end)
        else if ((uint32_t)(sl[q] >> 32) == (uint32_t)k[q]) m[q] = (uint32_t)sl[q];
        else m[q] = lookup(ks.table, ks.mask, k[q]);  // collision: probe on
      }
    }
    unsigned long long mine = 0;
    uint2* wf = flags + ((size_t)tile * kWarps + warp) * kOpItems;
#pragma unroll
    for (int q = 0; q < kOpItems; ++q) {
      const uint32_t once = __ballot_sync(0xFFFFFFFFu, m[q] != 0u);
      const uint32_t more = __ballot_sync(0xFFFFFFFFu, m[q] > 1u);
      if (lane == 0) wf[q] = make_uint2(once, more);
      mine += m[q];
    }
    mine = warp_sum(mine);
    if (lane == 0) s_w[buf][warp] = mine;
    __syncthreads();  // s_w[buf] is written again only after the next barrier
    if (tid == 0) {
      unsigned long long t = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t += s_w[buf][w];
      tile_cnt[tile] = t;
    }
  }
}

// tile_off[i] = cnt[0] + .. + cnt[i - 1] for i < ntiles, *total = the sum:
// blocks of 4096 counts (16 consecutive per thread), claimed in order, with
// the two-level decoupled look-back across blocks
__global__ void __launch_bounds__(kOpThreads)
    k_scan_counts(const uint64_t* __restrict__ cnt, uint32_t ntiles, uint64_t* __restrict__ tile_off,
                  OpScan sc, uint64_t* total) {
  __shared__ uint64_t s_sw[kOpThreads / 32 + 1];
  __shared__ uint32_t s_blk;
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x;
  if (tid == 0) s_blk = atomicAdd(sc.counter, 1u);
  __syncthreads();
  const uint32_t blk = s_blk;
  const uint32_t nblk = (ntiles + kOpTile - 1) / kOpTile;
  if (blk >= nblk) return;
  const uint32_t i0 = blk * kOpTile + (uint32_t)tid * kOpItems;
  uint64_t c[kOpItems], mine = 0;
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    c[q] = i0 + q < ntiles ? cnt[i0 + q] : 0ull;
    mine += c[q];
  }
  uint64_t btotal;
  uint64_t run = block_exclusive_sum<kOpThreads>(mine, s_sw, btotal);
  if (tid < 32) {
    const uint64_t excl = scan_prefix(sc.status, sc.ch, blk, nblk, btotal, sc.err);
    if (tid == 0) {
      s_prefix = excl;
      if (blk == nblk - 1) *total = excl + btotal;
    }
  }
  __syncthreads();
  run += s_prefix;
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    if (i0 + q < ntiles) tile_off[i0 + q] = run;
    run += c[q];
  }
}

// Join, writing pass: one block per tile (any order); a tile without output
// rows returns at once.  Rows are read only in the 32-row steps that have a
// match; each matching row is written once per occurrence of its key.
__global__ void __launch_bounds__(kOpThreads)
    k_join_write(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, uint32_t n,
                 int col, KeySet ks, const uint2* __restrict__ flags,
                 const uint64_t* __restrict__ tile_off, uint64_t total, int32_t* __restrict__ out_src,
                 int32_t* __restrict__ out_dst) {
  constexpr int kWarps = kOpThreads / 32;
  __shared__ uint32_t s_w[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blockIdx.x;
  const uint32_t ntiles = (n + kOpTile - 1) / kOpTile;
  const uint64_t t0 = tile_off[tile];
  const uint64_t t1 = tile + 1 < ntiles ? tile_off[tile + 1] : total;
  if (t0 == t1) return;
  const uint32_t base = tile * kOpTile + (uint32_t)warp * (32 * kOpItems) + (uint32_t)lane;
  const uint32_t lt = lanemask_lt();
  const uint2 myf = lane < kOpItems ? flags[((size_t)tile * kWarps + warp) * kOpItems + lane]
                                    : make_uint2(0u, 0u);
  int32_t s[kOpItems], d[kOpItems];
  uint32_t m[kOpItems];
  uint32_t wtotal = 0;
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t once = __shfl_sync(0xFFFFFFFFu, myf.x, q);
    const uint32_t more = __shfl_sync(0xFFFFFFFFu, myf.y, q);
    const uint32_t r = base + 32u * q;
    m[q] = 0u;
    s[q] = d[q] = 0;
    if ((once >> lane) & 1u) {
      s[q] = src[r];
      d[q] = dst[r];
      m[q] = ((more >> lane) & 1u) ? multiplicity(ks, col ? d[q] : s[q]) : 1u;
    }
    wtotal += more ? __reduce_add_sync(0xFFFFFFFFu, m[q]) : (uint32_t)__popc(once);
  }
  if (lane == 0) s_w[warp] = wtotal;
  __syncthreads();
  uint32_t w = (uint32_t)t0;  // the total fits 31 bits (checked before this pass)
  for (int k2 = 0; k2 < warp; ++k2) w += s_w[k2];
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t once = __shfl_sync(0xFFFFFFFFu, myf.x, q);
    const uint32_t more = __shfl_sync(0xFFFFFFFFu, myf.y, q);
    if (!more) {
      if ((once >> lane) & 1u) {
        const uint32_t p = w + __popc(once & lt);
        out_src[p] = s[q];
        out_dst[p] = d[q];
      }
      w += __popc(once);
    } else {
      const uint32_t inc = warp_inclusive_sum(m[q]);
      uint32_t p = w + inc - m[q];
      for (uint32_t t = 0; t < m[q]; ++t, ++p) {
        out_src[p] = s[q];
        out_dst[p] = d[q];
      }
      w += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
}

// Select, in place: one tile per block, claimed in order.  Warp w of the
// block owns rows [tile * 4096 + 512 w, + 512) and reads them 32 consecutive
// rows per step, so every load is one coalesced 128-byte line; a kept row's
// place among its warp's kept rows comes from a ballot per step.
__global__ void __launch_bounds__(kOpThreads)
    k_compact(int32_t* src, int32_t* dst, uint32_t n, int col, int op, int32_t value, OpScan sc,
              uint64_t* n_out) {
  constexpr int kWarps = kOpThreads / 32;
  __shared__ uint32_t s_sw[kWarps];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(sc.counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t ntiles = (n + kOpTile - 1) / kOpTile;
  if (tile >= ntiles) return;
  const uint32_t base = tile * kOpTile + (uint32_t)warp * (32 * kOpItems) + (uint32_t)lane;
  const uint32_t lt = lanemask_lt();
  int32_t s[kOpItems], d[kOpItems];
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    s[q] = r < n ? src[r] : 0;
    d[q] = r < n ? dst[r] : 0;
  }
  uint32_t wtotal = 0;  // kept rows of this warp
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    wtotal += __popc(__ballot_sync(0xFFFFFFFFu, r < n && compare(col ? d[q] : s[q], op, value)));
  }
  if (lane == 0) s_sw[warp] = wtotal;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < kWarps ? s_sw[lane] : 0u;
    const uint32_t inc = warp_inclusive_sum(t);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint64_t excl = scan_prefix(sc.status, sc.ch, tile, ntiles, (uint64_t)total, sc.err);
    if (lane < kWarps) s_sw[lane] = inc - t;
    if (lane == 0) {
      s_prefix = excl;
      if (tile == ntiles - 1) *n_out = excl + (uint64_t)total;
    }
  }
  __syncthreads();
  uint32_t w = (uint32_t)s_prefix + s_sw[warp];  // next output row of this warp
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    const bool keep = r < n && compare(col ? d[q] : s[q], op, value);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep) {
      const uint32_t p = w + __popc(b & lt);
      src[p] = s[q];
      dst[p] = d[q];
    }
    w += __popc(b);
  }
}

}  // namespace

// Scratch of one compaction run over n rows: statuses and chunk sums (zeroed)
struct CompactScratch {
  char* buf = nullptr;
  OpScan sc{};
  uint64_t* n_out = nullptr;
};

static int compact_scratch(uint32_t n, cudaStream_t s, CompactScratch* cs) {
  const uint64_t tiles = (n + kOpTile - 1) / kOpTile;
  const uint64_t chunks = (tiles + kChunkTiles - 1) / kChunkTiles;
  auto al = [](uint64_t x) { return (x + 255) & ~255ull; };
  const uint64_t bytes = al(8 * tiles) + 2 * al(8 * chunks) + al(4 * chunks) + al(64);
  char* b = (char*)pool_alloc(bytes, s);
  if (!b) return RINGO_ENOMEM;
  if (cudaMemsetAsync(b, 0, bytes, s) != cudaSuccess) {
    pool_free(b, s);
    return RINGO_ECUDA;
  }
  char* p = b;
  cs->buf = b;
  cs->sc.status = (uint64_t*)p;            p += al(8 * tiles);
  cs->sc.ch.agg = (uint64_t*)p;            p += al(8 * chunks);
  cs->sc.ch.inc = (uint64_t*)p;            p += al(8 * chunks);
  cs->sc.ch.cnt = (uint32_t*)p;            p += al(4 * chunks);
  cs->sc.err = (uint32_t*)p;
  cs->sc.counter = (uint32_t*)(p + 4);
  cs->n_out = (uint64_t*)(p + 8);
  return RINGO_OK;
}

int run_select(int32_t* src, int32_t* dst, uint32_t n, int col, int op, int32_t value,
               cudaStream_t s, uint64_t* n_out) {
  *n_out = 0;
  if (n == 0) return RINGO_OK;
  CompactScratch cs;
  if (int rc = compact_scratch(n, s, &cs)) return rc;
  const uint32_t tiles = (n + kOpTile - 1) / kOpTile;
  {
    ProfScope ps("select", s);
    k_compact<<<tiles, kOpThreads, 0, s>>>(src, dst, n, col, op, value, cs.sc, cs.n_out);
  }
  uint64_t h[2] = {0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, cs.n_out, 8, cudaMemcpyDeviceToHost, s);
  uint32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, cs.sc.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  pool_free(cs.buf, s);
  if (e != cudaSuccess) {
    set_error(std::string("select: ") + cudaGetErrorString(e));
    return RINGO_ECUDA;
  }
  if (herr) {
    set_error("select: a bounded device wait expired");
    return RINGO_ETIMEOUT;
  }
  *n_out = h[0];
  return RINGO_OK;
}

// The second table's key set (see KeySet); buffers in *owned, freed by the caller.
static int build_keyset(const int32_t* keys, uint32_t nkeys, cudaStream_t s, KeySet* ks,
                        std::vector<void*>* owned) {
  const uint32_t kg = (nkeys + 255) / 256 < 8192 ? (nkeys + 255) / 256 : 8192;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = pool_alloc(bytes, s);
    if (p) owned->push_back(p);
    return p;
  };
  auto hash_of = [&](uint64_t nk) -> uint32_t {  // slots for nk distinct keys, load <= 1/2
    uint32_t slots = 1;
    while (slots < 2 * nk) slots <<= 1;
    return slots;
  };
  *ks = KeySet{};
  const uint32_t slots = hash_of(nkeys);
  int32_t* mm = (int32_t*)alloc(256);
  if (!mm) return RINGO_ENOMEM;
  bool use_bits = false;
  int32_t hmm[2] = {0, 0};
  if (8ull * slots > kJoinHashCacheBytes) {
    // a bitmap when it is smaller than the hash table
    const int32_t init[2] = {0x7FFFFFFF, (int32_t)0x80000000};
    cudaError_t e = cudaMemcpyAsync(mm, init, 8, cudaMemcpyHostToDevice, s);
    k_key_range<<<kg, 256, 0, s>>>(keys, nkeys, mm);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmm, mm, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("join: ") + cudaGetErrorString(e));
      return RINGO_ECUDA;
    }
    const uint64_t range = (uint64_t)((int64_t)hmm[1] - (int64_t)hmm[0]) + 1;
    use_bits = 2 * 4 * ((range + 31) / 32) < 8ull * slots;
  }
  if (!use_bits) {
    unsigned long long* table = (unsigned long long*)alloc(8ull * slots);
    if (!table) return RINGO_ENOMEM;
    if (cudaMemsetAsync(table, 0, 8ull * slots, s) != cudaSuccess) return RINGO_ECUDA;
    {
      ProfScope ps("join_build", s);
      k_hash_build<<<kg, 256, 0, s>>>(keys, nkeys, table, slots - 1);
    }
    ks->table = table;
    ks->mask = slots - 1;
    return RINGO_OK;
  }
  const int64_t kmin = hmm[0];
  const uint64_t range = (uint64_t)((int64_t)hmm[1] - kmin) + 1;
  const size_t words = (size_t)((range + 31) / 32);
  uint32_t* bits = (uint32_t*)alloc(8 * words + 256);
  if (!bits) return RINGO_ENOMEM;
  uint32_t* dup = bits + words;
  unsigned long long* extra = (unsigned long long*)(dup + words);  // 8 * words bytes in: aligned
  unsigned long long hextra = 0;
  cudaError_t e = cudaMemsetAsync(bits, 0, 8 * words + 256, s);
  {
    ProfScope ps("join_build", s);
    k_bits_build<<<kg, 256, 0, s>>>(keys, nkeys, kmin, bits, dup, extra);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hextra, extra, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("join: ") + cudaGetErrorString(e));
    return RINGO_ECUDA;
  }
  ks->bits = bits;
  ks->kmin = kmin;
  ks->range = range;
  if (hextra) {  // at most hextra distinct keys repeat
    const uint32_t dslots = hash_of(hextra);
    unsigned long long* table = (unsigned long long*)alloc(8ull * dslots);
    if (!table) return RINGO_ENOMEM;
    if (cudaMemsetAsync(table, 0, 8ull * dslots, s) != cudaSuccess) return RINGO_ECUDA;
    {
      ProfScope ps("join_build", s);
      k_hash_dup<<<kg, 256, 0, s>>>(keys, nkeys, kmin, dup, table, dslots - 1);
    }
    ks->dup = dup;
    ks->table = table;
    ks->mask = dslots - 1;
  }
  return RINGO_OK;
}

int run_join(const int32_t* src, const int32_t* dst, uint32_t n, int col, const int32_t* keys,
             uint32_t nkeys, int32_t* out_src, int32_t* out_dst, uint64_t cap, cudaStream_t s,
             uint64_t* n_out) {
  *n_out = 0;
  if (n == 0 || nkeys == 0) return RINGO_OK;
  std::vector<void*> owned;
  auto done = [&](int rc) {
    for (void* p : owned) pool_free(p, s);
    return rc;
  };
  KeySet ks;
  if (int rc = build_keyset(keys, nkeys, s, &ks, &owned)) return done(rc);
  // marking pass: per-row flags and per-tile counts; then the tiles' offsets
  const uint32_t tiles = (n + kOpTile - 1) / kOpTile;
  uint2* flags = (uint2*)pool_alloc((size_t)tiles * kOpTile / 4 + 256, s);  // 2 bits per row
  if (!flags) return done(RINGO_ENOMEM);
  owned.push_back(flags);
  uint64_t* tile_cnt = (uint64_t*)pool_alloc(16ull * tiles + 256, s);
  if (!tile_cnt) return done(RINGO_ENOMEM);
  owned.push_back(tile_cnt);
  uint64_t* tile_off = tile_cnt + tiles;
  CompactScratch cs;
  if (int rc = compact_scratch(tiles, s, &cs)) return done(rc);
  owned.push_back(cs.buf);
  {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int mode = ks.bits ? kJoinBitmap : (ks.mask < kJoinSmemSlots ? kJoinSmemHash : kJoinHash);
    auto kern = mode == kJoinSmemHash ? k_join_mark<kJoinSmemHash>
                : mode == kJoinBitmap ? k_join_mark<kJoinBitmap>
                                      : k_join_mark<kJoinHash>;
    int per_sm = 0;  // persistent: the blocks that fit at once
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOpThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const uint64_t want = (uint64_t)sms * (uint64_t)per_sm;
    const uint32_t grid = tiles < want ? tiles : (uint32_t)want;
    ProfScope ps("join_mark", s);
    kern<<<grid, kOpThreads, 0, s>>>(col ? dst : src, n, ks, flags, tile_cnt);
    k_scan_counts<<<(tiles + kOpTile - 1) / kOpTile, kOpThreads, 0, s>>>(tile_cnt, tiles, tile_off,
                                                                        cs.sc, cs.n_out);
  }
  uint64_t htotal = 0;
  uint32_t herr = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&htotal, cs.n_out, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, cs.sc.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("join: ") + cudaGetErrorString(e));
    return done(RINGO_ECUDA);
  }
  if (herr) {
    set_error("join: a bounded device wait expired");
    return done(RINGO_ETIMEOUT);
  }
  *n_out = htotal;
  if (htotal > cap || htotal > 0x7FFFFFFFull) {
    set_error("join: the output has more rows than cap (or 2^31 - 1); nothing written");
    return done(RINGO_ERANGE);
  }
  if (htotal) {
    {
      ProfScope ps("join_write", s);
      k_join_write<<<tiles, kOpThreads, 0, s>>>(src, dst, n, col, ks, flags, tile_off, htotal,
                                                out_src, out_dst);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("join: ") + cudaGetErrorString(e));
      return done(RINGO_ECUDA);
    }
  }
  return done(RINGO_OK);
}

}  // namespace ringo

extern "C" {

int ringo_table_select(int32_t* src, int32_t* dst, int64_t nrows, int col, int op, int32_t value,
                       int64_t* n_out, void* stream) {
  if (!n_out) return RINGO_EINVAL;
  *n_out = 0;
  if (nrows < 0 || (nrows > 0 && (!src || !dst)) || (col != 0 && col != 1) || op < RINGO_CMP_LT ||
      op > RINGO_CMP_GT) {
    ringo::set_error("ringo_table_select: bad argument");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF) return RINGO_ERANGE;
  uint64_t k = 0;
  const int rc = ringo::run_select(src, dst, (uint32_t)nrows, col, op, value, (cudaStream_t)stream, &k);
  *n_out = (int64_t)k;
  return rc;
}

int ringo_table_join(const int32_t* src, const int32_t* dst, int64_t nrows, int col,
                     const int32_t* keys, int64_t nkeys, int32_t* out_src, int32_t* out_dst,
                     int64_t cap, int64_t* n_out, void* stream) {
  if (!n_out) return RINGO_EINVAL;
  *n_out = 0;
  if (nrows < 0 || nkeys < 0 || cap < 0 || (nrows > 0 && (!src || !dst)) || (nkeys > 0 && !keys) ||
      (col != 0 && col != 1)) {
    ringo::set_error("ringo_table_join: bad argument");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF || nkeys > 0x3FFFFFFF) return RINGO_ERANGE;
  if (cap > 0 && (!out_src || !out_dst)) return RINGO_EINVAL;
  uint64_t k = 0;
  const int rc = ringo::run_join(src, dst, (uint32_t)nrows, col, keys, (uint32_t)nkeys, out_src,
                                 out_dst, (uint64_t)cap, (cudaStream_t)stream, &k);
  *n_out = (int64_t)k;
  return rc;
}

}  // extern "C"
