// LSD radix sort of 64-bit keys for the table->graph conversion.
//
// The paper's conversion sorts copies of the source and destination columns
// (Section 3.4, sort-first).  Here both columns are sorted at once as packed
// 64-bit keys with a onesweep radix sort (Adinets & Merrill 2022): one kernel
// reads the columns once and builds the digit histograms of every pass; then
// each pass is a single kernel that ranks a 4096-key tile in shared memory
// with warp match/ballot digit counts, obtains its global digit offsets from
// a decoupled look-back over the tiles before it, and scatters the tile,
// staged in digit order in shared memory, with coalesced stores.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "device_util.cuh"
#include "ringo_internal.cuh"

namespace ringo {

// ---------------------------------------------------------------- K1 ------
// Digit histograms of all eight out-sort passes from one read of the columns.
// Pass p looks at bits [8p, 8p+8) of key = bias(src) << 32 | bias(dst).
constexpr int kHistThreads = 512;

__device__ __forceinline__ void hist_row(uint32_t (*h)[kRadix], int32_t s, int32_t d) {
  const uint32_t sb = (uint32_t)s ^ kBias, db = (uint32_t)d ^ kBias;
  atomicAdd(&h[0][db & 0xFF], 1u);
  atomicAdd(&h[1][(db >> 8) & 0xFF], 1u);
  atomicAdd(&h[2][(db >> 16) & 0xFF], 1u);
  atomicAdd(&h[3][db >> 24], 1u);
  atomicAdd(&h[4][sb & 0xFF], 1u);
  atomicAdd(&h[5][(sb >> 8) & 0xFF], 1u);
  atomicAdd(&h[6][(sb >> 16) & 0xFF], 1u);
  atomicAdd(&h[7][sb >> 24], 1u);
}

__global__ void __launch_bounds__(kHistThreads) k_histogram(Ctl* __restrict__ ctl) {
  __shared__ uint32_t h[kOutPasses][kRadix];
  for (int i = threadIdx.x; i < kOutPasses * kRadix; i += kHistThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int32_t* __restrict__ src = ctl->src;
  const int32_t* __restrict__ dst = ctl->dst;
  const uint32_t n = ctl->n_rows;
  const size_t stride = (size_t)gridDim.x * kHistThreads;
  const size_t t0 = (size_t)blockIdx.x * kHistThreads + threadIdx.x;
  const bool vec = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0;
  size_t done = 0;
  if (vec) {
    const size_t n4 = n / 4;
    const int4* s4 = reinterpret_cast<const int4*>(src);
    const int4* d4 = reinterpret_cast<const int4*>(dst);
    for (size_t i = t0; i < n4; i += stride) {
      const int4 a = __ldcs(s4 + i);
      const int4 b = __ldcs(d4 + i);
      hist_row(h, a.x, b.x);
      hist_row(h, a.y, b.y);
      hist_row(h, a.z, b.z);
      hist_row(h, a.w, b.w);
    }
    done = n4 * 4;
  }
  for (size_t i = done + t0; i < n; i += stride) hist_row(h, src[i], dst[i]);
  __syncthreads();

  for (int i = threadIdx.x; i < kOutPasses * kRadix; i += kHistThreads) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ctl->out_sort.hist[0][0] + i, c);
  }
}

void launch_histogram(Ctl* ctl, uint32_t n_rows, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t want = (n_rows + kHistThreads * 16 - 1) / (kHistThreads * 16);
  uint32_t grid = want < (uint32_t)sms * 4 ? want : (uint32_t)sms * 4;
  if (grid == 0) grid = 1;
  k_histogram<<<grid, kHistThreads, 0, s>>>(ctl);
}

// ---------------------------------------------------------------- plan ----
// Turns the pass histograms into global digit offsets and decides, on the
// device, which passes move keys: a pass whose digit is the same for every
// key is the identity and is skipped.  Also fixes the ping-pong buffers.
//   which = 0: out-sort of n_rows keys packed from the columns, digits at
//              bits 0..63 (passes 0-3: dst, 4-7: src); between pass 3 and
//              pass 4 the dst-rank step always runs (it also packs from the
//              columns when every dst pass was skipped); buffers keysA/keysB.
//   which = 1: in-sort of E keys held in the out-sort's spare buffer,
//              digits at bits 32..63 (the dst-run half).
__global__ void __launch_bounds__(kRadix) k_plan(Ctl* __restrict__ ctl, int which) {
  __shared__ uint32_t sw[kRadix / 32 + 1];
  __shared__ uint32_t trivial[kOutPasses];
  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const int npass = which ? kInPasses : kOutPasses;
  const uint32_t n = which ? ctl->E : ctl->n_rows;
  if (threadIdx.x < kOutPasses) trivial[threadIdx.x] = 0;
  __syncthreads();
  for (int p = 0; p < npass; ++p) {
    const uint32_t c = sc.hist[p][threadIdx.x];
    uint32_t total;
    const uint32_t excl = block_exclusive_sum<kRadix>(c, sw, total);
    sc.base[p][threadIdx.x] = excl;
    if (c == n) trivial[p] = 1;
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  sc.n = n;
  uint64_t* const b0 = which ? ctl->out_sort.spare : ctl->keysA;
  uint64_t* const b1 = which ? ctl->out_sort.result : ctl->keysB;
  const uint64_t* cur = which ? b0 : nullptr;
  uint64_t* next = which ? b1 : b0;
  uint32_t active = 0;
  const uint32_t shift0 = which ? 32 : 0;
  for (int p = 0; p < kOutPasses; ++p) {
    sc.pass[p].shift = shift0 + kRadixBits * p;
    sc.pass[p].active = 0;
    sc.pass[p].in = nullptr;
    sc.pass[p].out = nullptr;
  }
  for (int p = 0; p < npass; ++p) {
    if (which == 0 && p == 4) {
      ctl->rank_step.in = cur;
      ctl->rank_step.out = next;
      ctl->rank_step.active = 1;
      cur = next;
      next = (next == b0) ? b1 : b0;
    }
    if (trivial[p]) continue;
    sc.pass[p].active = 1;
    sc.pass[p].in = cur;
    sc.pass[p].out = next;
    cur = next;
    next = (next == b0) ? b1 : b0;
    ++active;
  }
  sc.active_passes = active;
  sc.result = const_cast<uint64_t*>(cur);
  sc.spare = (cur == b0) ? b1 : b0;
}

void launch_plan(Ctl* ctl, int which, cudaStream_t s) {
  k_plan<<<1, kRadix, 0, s>>>(ctl, which);
}

// ---------------------------------------------------------------- K2/K4 ---
// One onesweep LSD pass.  The kernel is persistent (a few blocks per SM) and
// walks tiles of kSortTile keys handed out in order by an atomic counter.
// Each tile arrives in shared memory by bulk asynchronous copy
// (cp.async.bulk + mbarrier) into one of two buffers, so the next tile's
// load is in flight while the current one is ranked, looked back and
// scattered.  Per tile:
//   1. every warp ranks its 512 keys in position order: match.any finds the
//      lanes holding the same digit, the highest of them bumps the warp's
//      digit counter for the group;
//   2. thread d owns digit d: it sums the warp counters, publishes the
//      tile's digit count, and obtains the count of digit d in all earlier
//      tiles by decoupled look-back (bounded waits);
//   3. the tile is re-staged in digit order in the same buffer and written
//      out with consecutive keys of a digit going to consecutive addresses.
// which: 0 out-sort, 1 in-sort.  pass: index within that sort.  gpass: global
// pass number; status region gpass&1 is used, and every processed tile clears
// its row of region (gpass+1)&1 for the next pass.  Tiles are claimed in
// increasing order and a tile waits only on smaller tiles, every one of which
// is held by a running block that never waits on a larger tile, so the
// waits always end.

// Decoupled look-back for one digit: the count of digit `d` in tiles
// [0, tile).  Reads kLookWindow predecessor statuses per round trip, adding
// aggregates until it meets an inclusive prefix; an unpublished status is
// re-polled with backoff.  Bounded: gives up after kSpinLimit polls, or once
// another block has recorded an error.
constexpr int kLookWindow = 16;
__device__ __forceinline__ uint32_t digit_lookback(const uint32_t* __restrict__ st,
                                                   uint32_t tile, uint32_t d, Ctl* ctl) {
  uint32_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  uint32_t spins = 0;
  const volatile uint32_t* verr = &ctl->err;
  while (j >= 0) {
    uint32_t v[kLookWindow];
#pragma unroll
    for (int k = 0; k < kLookWindow; ++k)
      v[k] = (j - k >= 0) ? ld_relaxed_u32(st + (size_t)(j - k) * kRadix + d) : kStInc;
    int k = 0;
    bool done = false;
#pragma unroll
    for (int q = 0; q < kLookWindow; ++q) {
      if (done || k != q) continue;
      const uint32_t x = v[q];
      if (x == 0) continue;  // not yet published: stop here
      if (x & kStInc) {
        excl += x & ~kStInc;
        done = true;
      } else {
        excl += x - 1u;
        k = q + 1;
      }
    }
    if (done) break;
    j -= k;
    if (k < kLookWindow) {
      if (spin_backoff(spins) || ((spins & 255) == 0 && *verr)) {
        atomicOr(&ctl->err, kErrLookback);
        break;
      }
    }
  }
  return excl;
}

struct SweepSmem {
  uint64_t buf[2][kSortTile];
  uint32_t whist[kSortWarps][kRadix];
  int32_t delta[kRadix];
  uint32_t binstart[kRadix];
  uint32_t sw[kSortWarps + 1];
  uint32_t next_tile[2];
  uint32_t bulk_cnt[2];
  uint32_t ok;
  uint64_t bar[2];
};

__device__ __forceinline__ void sweep_issue(SweepSmem& S, int b, uint32_t tile, uint32_t n,
                                            const uint64_t* in, const int32_t* src,
                                            const int32_t* dst, bool cols_bulk) {
  const uint32_t base = tile * (uint32_t)kSortTile;
  const uint32_t cnt = min((uint32_t)kSortTile, n - base);
  uint32_t bulk, bytes;
  if (in) {
    bulk = cnt & ~1u;                    // 8-byte keys: an even count is 16-byte sized
    bytes = bulk * 8u;
  } else if (cols_bulk) {
    bulk = cnt & ~3u;                    // 4-byte IDs: a multiple of 4
    bytes = bulk * 8u;                   // both columns
  } else {
    bulk = 0;
    bytes = 0;
  }
  S.bulk_cnt[b] = bulk;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&S.bar[b], bytes);
  if (bulk) {
    if (in) {
      bulk_g2s(&S.buf[b][0], in + base, bulk * 8u, &S.bar[b]);
    } else {
      int32_t* cols = reinterpret_cast<int32_t*>(&S.buf[b][0]);
      bulk_g2s(cols, src + base, bulk * 4u, &S.bar[b]);
      bulk_g2s(cols + kSortTile, dst + base, bulk * 4u, &S.bar[b]);
    }
  }
}

__global__ void __launch_bounds__(kSortThreads, 2)
    k_onesweep_persistent(Ctl* __restrict__ ctl, int which, int pass, int gpass) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SweepSmem& S = *reinterpret_cast<SweepSmem*>(smem_raw);
  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const PassDesc pd = sc.pass[pass];
  const uint32_t n = sc.n;
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* __restrict__ st_next = ctl->status[(gpass + 1) & 1];
  if (!pd.active) {
    const size_t rows = (size_t)ntiles * kRadix;
    for (size_t i = (size_t)blockIdx.x * kSortThreads + tid; i < rows;
         i += (size_t)gridDim.x * kSortThreads)
      st_next[i] = 0;
    return;
  }
  uint32_t* __restrict__ st = ctl->status[gpass & 1];
  const uint64_t* __restrict__ in = pd.in;
  const int32_t* __restrict__ src = ctl->src;
  const int32_t* __restrict__ dst = ctl->dst;
  const bool cols_bulk = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0;
  const uint32_t shift = pd.shift;
  uint64_t* __restrict__ out = pd.out;
  const volatile uint32_t* verr = &ctl->err;

  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    mbar_init_fence();
    const uint32_t t0 = atomicAdd(&sc.tile_counter[pass], 1u);
    S.next_tile[0] = t0;
    if (t0 < ntiles) sweep_issue(S, 0, t0, n, in, src, dst, cols_bulk);
  }
  __syncthreads();
  uint32_t tile = S.next_tile[0];
  int b = 0;
  uint32_t phase0 = 0, phase1 = 0;
  while (tile < ntiles) {
    // claim the next tile and start its load into the other buffer
    if (tid == 0) {
      const uint32_t nt = atomicAdd(&sc.tile_counter[pass], 1u);
      S.next_tile[b ^ 1] = nt;
      if (nt < ntiles) sweep_issue(S, b ^ 1, nt, n, in, src, dst, cols_bulk);
    }
    st_next[(size_t)tile * kRadix + tid] = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) S.whist[w][tid] = 0;
    const uint32_t base = tile * (uint32_t)kSortTile;
    const uint32_t cnt = min((uint32_t)kSortTile, n - base);
    {
      // thread 0 waits (bounded) and tells the block; the others then see a
      // completed phase at once
      const uint32_t par = b ? phase1 : phase0;
      if (tid == 0) S.ok = mbar_wait_bounded(&S.bar[b], par, verr) ? 1u : 0u;
      __syncthreads();
      if (!S.ok) {
        if (tid == 0) {
          atomicOr(&ctl->err, kErrLookback);
          // let this block's own copies land before it exits
          mbar_wait_bounded(&S.bar[b], par, nullptr);
          if (S.next_tile[b ^ 1] < ntiles)
            mbar_wait_bounded(&S.bar[b ^ 1], b ? phase0 : phase1, nullptr);
        }
        return;
      }
      while (!mbar_try_wait(&S.bar[b], par)) {
      }
      if (b) phase1 ^= 1u; else phase0 ^= 1u;
    }
    // the part of the tile the bulk copy did not cover (ragged tail or
    // unaligned columns) comes in with plain loads
    const uint32_t bulk = S.bulk_cnt[b];
    if (in) {
      for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) S.buf[b][j] = in[base + j];
    } else {
      int32_t* cols = reinterpret_cast<int32_t*>(&S.buf[b][0]);
      for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) {
        cols[j] = src[base + j];
        cols[kSortTile + j] = dst[base + j];
      }
    }
    __syncthreads();

    // keys into registers, warp-striped: item i of lane l is tile slot
    // 512 warp + 32 i + l
    uint64_t key[kSortItems];
    uint32_t valid = 0;
    const uint32_t wslot = warp * (kSortItems * 32);
    if (in) {
#pragma unroll
      for (int i = 0; i < kSortItems; ++i) {
        const uint32_t j = wslot + i * 32 + lane;
        key[i] = S.buf[b][j];
        if (j < cnt) valid |= 1u << i;
      }
    } else {
      const int32_t* cols = reinterpret_cast<const int32_t*>(&S.buf[b][0]);
#pragma unroll
      for (int i = 0; i < kSortItems; ++i) {
        const uint32_t j = wslot + i * 32 + lane;
        const uint32_t sb = (uint32_t)cols[j] ^ kBias;
        const uint32_t db = (uint32_t)cols[kSortTile + j] ^ kBias;
        key[i] = ((uint64_t)sb << 32) | db;
        if (j < cnt) valid |= 1u << i;
      }
    }
    uint16_t rank[kSortItems];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const bool ok = (valid >> i) & 1u;
      const uint32_t dig = ok ? (uint32_t)(key[i] >> shift) & (kRadix - 1) : kRadix;
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
      const int leader = 31 - __clz(peers);
      uint32_t old = 0;
      if (lane == leader && ok) old = atomicAdd(&S.whist[warp][dig], (uint32_t)__popc(peers));
      old = __shfl_sync(0xFFFFFFFFu, old, leader);
      rank[i] = (uint16_t)(old + __popc(peers & lt));
    }
    __syncthreads();

    uint32_t bin_total = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = S.whist[w][tid];
      S.whist[w][tid] = bin_total;
      bin_total += c;
    }
    uint32_t* my_st = st + (size_t)tile * kRadix + tid;
    st_relaxed_u32(my_st, tile == 0 ? (kStInc | bin_total) : (1u + bin_total));
    uint32_t tile_total;
    const uint32_t bin_start = block_exclusive_sum<kSortThreads>(bin_total, S.sw, tile_total);
    S.binstart[tid] = bin_start;
    uint32_t excl = 0;
    if (tile > 0) {
      excl = digit_lookback(st, tile, tid, ctl);
      st_relaxed_u32(my_st, kStInc | (excl + bin_total));
    }
    S.delta[tid] = (int32_t)(sc.base[pass][tid] + excl) - (int32_t)bin_start;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      if ((valid >> i) & 1u) {
        const uint32_t dig = (uint32_t)(key[i] >> shift) & (kRadix - 1);
        S.buf[b][S.binstart[dig] + S.whist[warp][dig] + rank[i]] = key[i];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (uint32_t j = tid; j < cnt; j += kSortThreads) {
      const uint64_t k = S.buf[b][j];
      const uint32_t dig = (uint32_t)(k >> shift) & (kRadix - 1);
      out[(uint32_t)(S.delta[dig] + (int32_t)j)] = k;
    }
    fence_proxy_async_smem();  // this buffer is the target of a later bulk copy
    __syncthreads();
    tile = S.next_tile[b ^ 1];
    b ^= 1;
  }
}


// Lanes of the warp whose 8-bit digit (plus a validity bit) equals this
// lane's: nine ballots, one per bit, each kept or inverted by the lane's own
// bit.
__device__ __forceinline__ uint32_t digit_peers(uint32_t dig, bool ok) {
  uint32_t peers = ok ? __ballot_sync(0xFFFFFFFFu, ok) : ~__ballot_sync(0xFFFFFFFFu, ok);
#pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const bool bit = (dig >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// The same pass with one tile per block: several blocks per SM overlap
// their phases.  Digit counts are taken first and published at once (so
// later tiles find them already visible when they look back), then keys are
// ranked with ballot-built peer masks, then the look-back runs.
__global__ void __launch_bounds__(kSortThreads, 3)
    k_onesweep_blocked(Ctl* __restrict__ ctl, int which, int pass, int gpass) {
  __shared__ uint64_t s_keys[kSortTile];
  __shared__ uint32_t s_whist[kSortWarps][kRadix];
  __shared__ int32_t s_delta[kRadix];
  __shared__ uint32_t s_binstart[kRadix];
  __shared__ uint32_t s_sw[kSortWarps + 1];
  __shared__ uint32_t s_tile;

  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(&sc.tile_counter[pass], 1u);
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) s_whist[w][tid] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile < ctl->status_rows)
    ctl->status[(gpass + 1) & 1][(size_t)tile * kRadix + tid] = 0;
  const PassDesc pd = sc.pass[pass];
  const uint32_t n = sc.n;
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  if (!pd.active || tile >= ntiles) return;
  uint32_t* __restrict__ st = ctl->status[gpass & 1];
  const uint32_t base = tile * (uint32_t)kSortTile;
  const uint32_t wbase = base + warp * (kSortItems * 32);
  const uint32_t shift = pd.shift;

  uint64_t key[kSortItems];
  uint32_t valid = 0;
  if (pd.in) {
    const uint64_t* __restrict__ in = pd.in;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const uint32_t pos = wbase + i * 32 + lane;
      if (pos < n) {
        key[i] = __ldcs(in + pos);
        valid |= 1u << i;
      } else {
        key[i] = 0;
      }
    }
  } else {
    const int32_t* __restrict__ src = ctl->src;
    const int32_t* __restrict__ dst = ctl->dst;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const uint32_t pos = wbase + i * 32 + lane;
      if (pos < n) {
        const uint32_t sb = (uint32_t)__ldcs(src + pos) ^ kBias;
        const uint32_t db = (uint32_t)__ldcs(dst + pos) ^ kBias;
        key[i] = ((uint64_t)sb << 32) | db;
        valid |= 1u << i;
      } else {
        key[i] = 0;
      }
    }
  }
  // 1. digit counts per warp (shared-memory reductions, no return values)
#pragma unroll
  for (int i = 0; i < kSortItems; ++i)
    if ((valid >> i) & 1u) atomicAdd(&s_whist[warp][(uint32_t)(key[i] >> shift) & (kRadix - 1)], 1u);
  __syncthreads();
  // 2. thread tid owns digit tid: warp prefixes, tile count, publish
  uint32_t bin_total = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = s_whist[w][tid];
    s_whist[w][tid] = bin_total;
    bin_total += c;
  }
  uint32_t* my_st = st + (size_t)tile * kRadix + tid;
  st_relaxed_u32(my_st, tile == 0 ? (kStInc | bin_total) : (1u + bin_total));
  uint32_t tile_total;
  const uint32_t bin_start = block_exclusive_sum<kSortThreads>(bin_total, s_sw, tile_total);
  s_binstart[tid] = bin_start;
  __syncthreads();
  // 3. stable ranks: within a warp, position order is (item, lane); the
  //    highest peer advances the warp's running offset for the digit
  uint16_t lpos[kSortItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const bool ok = (valid >> i) & 1u;
    const uint32_t dig = (uint32_t)(key[i] >> shift) & (kRadix - 1);
    const uint32_t peers = digit_peers(dig, ok);
    const int leader = 31 - __clz(peers);
    uint32_t old = 0;
    if (lane == leader && ok) old = atomicAdd(&s_whist[warp][dig], (uint32_t)__popc(peers));
    old = __shfl_sync(0xFFFFFFFFu, old, leader);
    lpos[i] = (uint16_t)(s_binstart[dig] + old + __popc(peers & lt));
  }
  // 4. look-back for the digit's offset in earlier tiles
  uint32_t excl = 0;
  if (tile > 0) {
    excl = digit_lookback(st, tile, tid, ctl);
    st_relaxed_u32(my_st, kStInc | (excl + bin_total));
  }
  s_delta[tid] = (int32_t)(sc.base[pass][tid] + excl) - (int32_t)bin_start;
  // 5. stage in digit order, then write out
#pragma unroll
  for (int i = 0; i < kSortItems; ++i)
    if ((valid >> i) & 1u) s_keys[lpos[i]] = key[i];
  __syncthreads();
  const uint32_t nvalid = min((uint32_t)kSortTile, n - base);
  uint64_t* __restrict__ out = pd.out;
#pragma unroll 4
  for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
    const uint64_t k = s_keys[j];
    const uint32_t dig = (uint32_t)(k >> shift) & (kRadix - 1);
    out[(uint32_t)(s_delta[dig] + (int32_t)j)] = k;
  }
}

static int g_sweep_blocks_per_sm = 0;
static int g_sweep_variant = -1;  // 0: one tile per block, 1: persistent

int onesweep_variant() {
  if (g_sweep_variant < 0) {
    const char* v = getenv("RINGO_ONESWEEP");
    g_sweep_variant = (v && v[0] == 'p') ? 1 : 0;
  }
  return g_sweep_variant;
}

void launch_onesweep(Ctl* ctl, int which, int pass, int gpass, uint32_t tiles, cudaStream_t s) {
  if (tiles == 0) return;
  if (onesweep_variant() == 0) {
    k_onesweep_blocked<<<tiles, kSortThreads, 0, s>>>(ctl, which, pass, gpass);
    return;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_sweep_blocks_per_sm == 0) {
    cudaFuncSetAttribute(k_onesweep_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SweepSmem));
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_onesweep_persistent, kSortThreads,
                                                  sizeof(SweepSmem));
    g_sweep_blocks_per_sm = per > 0 ? per : 1;
  }
  uint32_t grid = (uint32_t)sms * (uint32_t)g_sweep_blocks_per_sm;
  if (grid > tiles) grid = tiles;
  k_onesweep_persistent<<<grid, kSortThreads, sizeof(SweepSmem), s>>>(ctl, which, pass, gpass);
}

}  // namespace ringo
