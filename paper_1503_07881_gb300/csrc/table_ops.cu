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
// is read.  Join builds an open-addressing hash table of the second table's
// keys with their multiplicities first.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kOpThreads = 256;
constexpr uint32_t kOpItems = 16;
constexpr uint32_t kOpTile = kOpThreads * kOpItems;  // 4096 rows

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
__device__ __forceinline__ uint32_t lookup(const unsigned long long* __restrict__ table, uint32_t mask,
                                           int32_t k) {
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

// total output rows of the join (64-bit), to size and check it before writing
__global__ void k_join_count(const int32_t* __restrict__ keycol, uint32_t n,
                             const unsigned long long* __restrict__ table, uint32_t mask,
                             unsigned long long* __restrict__ total) {
  unsigned long long c = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    c += lookup(table, mask, keycol[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}

// One tile of the compaction.  kMode 0: select (in place, src/dst are both
// input and output); kMode 1: join (each row written mult times into out).
// Warp w of the block owns rows [tile * 4096 + 512 w, + 512) and reads them
// 32 consecutive rows per step, so every load is one coalesced 128-byte
// line; a row's place among the warp's output rows comes from a ballot
// (select) or a warp scan of multiplicities (join) per step.
template <int kMode>
__global__ void __launch_bounds__(kOpThreads)
    k_compact(int32_t* src, int32_t* dst, uint32_t n, int col, int op, int32_t value,
              const unsigned long long* __restrict__ table, uint32_t mask,
              int32_t* __restrict__ out_src, int32_t* __restrict__ out_dst, OpScan sc,
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
  uint32_t m[kMode == 0 ? 1 : kOpItems];
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    s[q] = r < n ? src[r] : 0;
    d[q] = r < n ? dst[r] : 0;
  }
  uint32_t wtotal = 0;  // output rows of this warp
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    const int32_t key = col ? d[q] : s[q];
    if constexpr (kMode == 0) {
      wtotal += __popc(__ballot_sync(0xFFFFFFFFu, r < n && compare(key, op, value)));
    } else {
      m[q] = r < n ? lookup(table, mask, key) : 0u;
      wtotal += __reduce_add_sync(0xFFFFFFFFu, m[q]);
    }
  }
  if (lane == 0) s_sw[warp] = wtotal;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < kWarps ? s_sw[lane] : 0u;
    const uint32_t inc = warp_inclusive_sum(t);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint64_t excl = scan_prefix(sc.status, sc.ch, tile, ntiles, pack2(0, total), sc.err);
    if (lane < kWarps) s_sw[lane] = inc - t;
    if (lane == 0) {
      s_prefix = excl;
      if (tile == ntiles - 1) *n_out = unpackB(excl) + (uint64_t)total;
    }
  }
  __syncthreads();
  uint32_t w = (uint32_t)unpackB(s_prefix) + s_sw[warp];  // next output row of this warp
  int32_t* os = kMode == 0 ? src : out_src;
  int32_t* od = kMode == 0 ? dst : out_dst;
#pragma unroll
  for (int q = 0; q < kOpItems; ++q) {
    const uint32_t r = base + 32u * q;
    const int32_t key = col ? d[q] : s[q];
    if constexpr (kMode == 0) {
      const bool keep = r < n && compare(key, op, value);
      const uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const uint32_t p = w + __popc(b & lt);
        os[p] = s[q];
        od[p] = d[q];
      }
      w += __popc(b);
    } else {
      const uint32_t inc = warp_inclusive_sum(m[q]);
      uint32_t p = w + inc - m[q];
      for (uint32_t t = 0; t < m[q]; ++t, ++p) {
        os[p] = s[q];
        od[p] = d[q];
      }
      w += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
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
    k_compact<0><<<tiles, kOpThreads, 0, s>>>(src, dst, n, col, op, value, nullptr, 0, nullptr,
                                              nullptr, cs.sc, cs.n_out);
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

int run_join(const int32_t* src, const int32_t* dst, uint32_t n, int col, const int32_t* keys,
             uint32_t nkeys, int32_t* out_src, int32_t* out_dst, uint64_t cap, cudaStream_t s,
             uint64_t* n_out) {
  *n_out = 0;
  if (n == 0 || nkeys == 0) return RINGO_OK;
  uint32_t slots = 1;
  while (slots < 2u * nkeys) slots <<= 1;  // load factor at most 1/2
  const uint32_t mask = slots - 1;
  unsigned long long* table = (unsigned long long*)pool_alloc(8ull * slots + 256, s);
  if (!table) return RINGO_ENOMEM;
  unsigned long long* total = table + slots;
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(table, 0, 8ull * slots + 8, s);
  const uint32_t kg = (nkeys + 255) / 256 < 8192 ? (nkeys + 255) / 256 : 8192;
  const uint32_t ng = (n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192;
  unsigned long long htotal = 0;
  {
    ProfScope ps("join_build", s);
    k_hash_build<<<kg, 256, 0, s>>>(keys, nkeys, table, mask);
  }
  {
    ProfScope ps("join_count", s);
    k_join_count<<<ng, 256, 0, s>>>(col ? dst : src, n, table, mask, total);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&htotal, total, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("join: ") + cudaGetErrorString(e));
    pool_free(table, s);
    return RINGO_ECUDA;
  }
  *n_out = htotal;
  if (htotal > cap || htotal > 0x7FFFFFFFull) {
    set_error("join: the output has more rows than cap (or 2^31 - 1); nothing written");
    pool_free(table, s);
    return RINGO_ERANGE;
  }
  if (htotal) {
    CompactScratch cs;
    rc = compact_scratch(n, s, &cs);
    if (rc == RINGO_OK) {
      const uint32_t tiles = (n + kOpTile - 1) / kOpTile;
      {
        ProfScope ps("join_write", s);
        k_compact<1><<<tiles, kOpThreads, 0, s>>>(const_cast<int32_t*>(src),
                                                  const_cast<int32_t*>(dst), n, col, 0, 0, table,
                                                  mask, out_src, out_dst, cs.sc, cs.n_out);
      }
      uint32_t herr = 0;
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, cs.sc.err, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error(std::string("join: ") + cudaGetErrorString(e));
        rc = RINGO_ECUDA;
      } else if (herr) {
        set_error("join: a bounded device wait expired");
        rc = RINGO_ETIMEOUT;
      }
      pool_free(cs.buf, s);
    }
  }
  pool_free(table, s);
  return rc;
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
