// LSD radix sort of 64-bit keys for the table->graph conversion.
//
// The paper's conversion sorts copies of the source and destination columns
// (Section 3.4, sort-first).  Here both columns are sorted at once as packed
// 64-bit keys with onesweep radix passes (Adinets & Merrill 2022): one kernel
// reads the columns once and builds the digit histograms of every pass; then
// each pass is a single kernel that brings a 4096-key tile into shared memory
// with a bulk asynchronous copy, counts and ranks its digits with warp-level
// peer masks, obtains the global digit offsets from a two-level decoupled
// look-back (tiles within a 32-tile chunk, then chunk aggregates), and
// scatters the tile, staged in digit order, with coalesced stores.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>


#include "device_util.cuh"
#include "ringo_internal.cuh"

namespace ringo {

// ---------------------------------------------------------------- K1 ------
// Digit histograms of all eight out-sort passes from one read of the columns.
// Pass p looks at bits [8p, 8p+8) of key = bias(src) << 32 | bias(dst).
// Persistent blocks claim 4096-row tiles in order and keep a shared
// histogram while the tiles belong to one segment, adding it to that
// segment's control block when the segment changes and at the end.
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

__global__ void __launch_bounds__(kHistThreads)
    k_histogram(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ uint32_t h[kOutPasses][kRadix];
  __shared__ Claim cl;
  __shared__ uint32_t cur_seg;
  for (int i = threadIdx.x; i < kOutPasses * kRadix; i += kHistThreads) (&h[0][0])[i] = 0;
  if (threadIdx.x == 0) cur_seg = 0xFFFFFFFFu;
  auto flush = [&](uint32_t sidx) {
    uint32_t* dst = &ctls[sidx].out_sort.hist[0][0];
    for (int i = threadIdx.x; i < kOutPasses * kRadix; i += kHistThreads) {
      const uint32_t c = (&h[0][0])[i];
      if (c) {
        atomicAdd(dst + i, c);
        (&h[0][0])[i] = 0;
      }
    }
  };
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) claim_slot(m, counter, &cl);
    __syncthreads();
    if (!cl.valid) break;
    if (cl.seg != cur_seg) {
      if (cur_seg != 0xFFFFFFFFu) flush(cur_seg);
      __syncthreads();
      if (threadIdx.x == 0) cur_seg = cl.seg;
    }
    const Ctl* ctl = ctls + cl.seg;
    const uint32_t n = ctl->n_rows;
    const uint32_t base = cl.tile * (uint32_t)kSortTile;
    if (base >= n) continue;
    const uint32_t cnt = min((uint32_t)kSortTile, n - base);
    const int32_t* __restrict__ src = ctl->src + base;
    const int32_t* __restrict__ dst = ctl->dst + base;
    const bool vec = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0;
    uint32_t done = 0;
    if (vec) {
      const uint32_t n4 = cnt / 4;
      for (uint32_t i = threadIdx.x; i < n4; i += kHistThreads) {
        const int4 a = __ldcs(reinterpret_cast<const int4*>(src) + i);
        const int4 b = __ldcs(reinterpret_cast<const int4*>(dst) + i);
        hist_row(h, a.x, b.x);
        hist_row(h, a.y, b.y);
        hist_row(h, a.z, b.z);
        hist_row(h, a.w, b.w);
      }
      done = n4 * 4;
    }
    for (uint32_t i = done + threadIdx.x; i < cnt; i += kHistThreads) hist_row(h, src[i], dst[i]);
  }
  __syncthreads();
  if (cur_seg != 0xFFFFFFFFu) flush(cur_seg);
}

void launch_histogram(const Launch& L, uint32_t* counter, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t grid = (uint32_t)sms * 4;
  if (grid > L.row_slots) grid = L.row_slots;
  if (grid == 0) return;
  k_histogram<<<grid, kHistThreads, 0, s>>>(L.ctls, L.rows, counter);
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
__global__ void __launch_bounds__(kRadix) k_plan(Ctl* __restrict__ ctls, int which) {
  Ctl* __restrict__ ctl = ctls + blockIdx.x;
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

void launch_plan(const Launch& L, int which, cudaStream_t s) {
  if (L.nseg) k_plan<<<L.nseg, kRadix, 0, s>>>(L.ctls, which);
}

// ---------------------------------------------------------------- K2/K4 ---
// One onesweep LSD pass: one block per tile of kSortTile keys, tiles claimed
// in increasing order through an atomic counter (the kernel and its per-tile
// steps are described at k_onesweep below).  which: 0 out-sort, 1 in-sort.
// pass: index within that sort.  gpass: global pass number; status region
// gpass&1 is used, and every processed tile clears its row of region
// (gpass+1)&1 for the next pass.  A tile waits only on smaller tiles, every
// one of which was claimed by a block that is resident or done and never
// waits on a larger tile, so the waits always end.

// Two-level decoupled look-back for digit d of `tile`: first over the
// earlier tiles of the tile's own chunk (their aggregates or an inclusive
// prefix), then over earlier chunks: a chunk whose tiles have all added their
// counts contributes its aggregate, a chunk whose inclusive prefix is known
// ends the walk.  A chunk's aggregate is complete soon after its tiles have
// counted, so no wait follows the chain of inclusive prefixes tile by tile.
// Bounded like every wait here.
__device__ __forceinline__ uint32_t digit_lookback2(const uint32_t* __restrict__ st,
                                                    const uint32_t* __restrict__ cagg,
                                                    const uint32_t* __restrict__ cinc,
                                                    const uint32_t* __restrict__ ccnt,
                                                    uint32_t tile, uint32_t ntiles, uint32_t d,
                                                    Ctl* ctl) {
  constexpr int W = kChunkTiles / 2;
  const volatile uint32_t* verr = &ctl->err;
  uint32_t excl = 0, spins = 0;
  const uint32_t c = tile >> kChunkShift;
  const uint32_t first = c << kChunkShift;
  // 1. tiles [first, tile) of this chunk
  int64_t j = (int64_t)tile - 1;
  while (j >= (int64_t)first) {
    uint32_t v[W];
#pragma unroll
    for (int k = 0; k < W; ++k)
      v[k] = (j - k >= (int64_t)first) ? ld_relaxed_u32(st + (size_t)(j - k) * kRadix + d) : 0u;
    int used = 0;
    bool done = false, stall = false;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      if (done || stall || j - q < (int64_t)first) continue;
      const uint32_t x = v[q];
      if (x == 0) {
        stall = true;
      } else if (x & kStInc) {
        excl += x & ~kStInc;
        done = true;
      } else {
        excl += x - 1u;
        used = q + 1;
      }
    }
    if (done) return excl;
    j -= used;
    if (stall) {
      if (spin_backoff(spins) || ((spins & 255) == 0 && *verr)) {
        atomicOr(&ctl->err, kErrLookback);
        return excl;
      }
    }
  }
  // 2. chunks c-1, c-2, ...
  int64_t cc = (int64_t)c - 1;
  while (cc >= 0) {
    const uint32_t inc = ld_relaxed_u32(cinc + (size_t)cc * kRadix + d);
    if (inc & kStInc) return excl + (inc & ~kStInc);
    const uint32_t cnt = ld_acquire_u32(ccnt + cc);
    const uint32_t need = min((uint32_t)kChunkTiles, ntiles - ((uint32_t)cc << kChunkShift));
    if (cnt >= need) {
      excl += ld_relaxed_u32(cagg + (size_t)cc * kRadix + d);
      --cc;
      continue;
    }
    if (spin_backoff(spins) || ((spins & 255) == 0 && *verr)) {
      atomicOr(&ctl->err, kErrLookback);
      return excl;
    }
  }
  return excl;
}

// The pass as used by default.  One 4096-key tile per block, four blocks per
// SM.  Per tile:
//   0. the tile arrives in shared memory by one bulk asynchronous copy
//      (cp.async.bulk + mbarrier; the first pass copies the two columns);
//   1. digit counts per warp (shared-memory reductions), published at once,
//      also into the chunk aggregate of the two-level look-back;
//   2. warp offsets within each digit plus the tile's digit starts;
//   3. ranks: the lanes of a warp holding the same digit find each other
//      through a shared peer mask (atomicOr of lane bits), the highest of
//      them advances the warp's digit offset for the group;
//   4. the keys move to their ranked places in the same buffer;
//   5. two-level look-back;
//   6. coalesced scatter of the staged tile.
// Keys sit in registers only during step 4, so a block needs few registers.
struct SweepV6Smem {
  uint64_t keys[kSortTile];               // the tile: input, then staged in digit order
  uint32_t whist[kSortWarps][kRadix];
  uint32_t mask[kSortWarps][kRadix + 1];  // slot kRadix: lanes past the end
  int32_t delta[kRadix];
  uint32_t sw[kSortWarps + 1];
  Claim claim;
  uint32_t ok;
  uint64_t bar;
};

__global__ void __launch_bounds__(kSortThreads, 4)
    k_onesweep(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter, int which, int pass,
               int gpass) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SweepV6Smem& S = *reinterpret_cast<SweepV6Smem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    claim_slot(m, counter, &S.claim);
    mbar_init(&S.bar, 1);
    mbar_init_fence();
  }
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    S.whist[w][tid] = 0;
    S.mask[w][tid] = 0;
  }
  if (tid < kSortWarps) S.mask[tid][kRadix] = 0;
  __syncthreads();
  if (!S.claim.valid) return;
  Ctl* __restrict__ ctl = ctls + S.claim.seg;
  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const uint32_t tile = S.claim.tile;
  const int reg = gpass & 1, nreg = reg ^ 1;
  if (tile < ctl->status_rows) {
    // clear this tile's row (and, for a chunk's first tile, the chunk's row)
    // of the other region for the next pass
    ctl->status[nreg][(size_t)tile * kRadix + tid] = 0;
    if ((tile & (kChunkTiles - 1)) == 0) {
      const uint32_t cidx = tile >> kChunkShift;
      ctl->chunk_agg[nreg][(size_t)cidx * kRadix + tid] = 0;
      ctl->chunk_inc[nreg][(size_t)cidx * kRadix + tid] = 0;
      if (tid == 0) ctl->chunk_cnt[nreg][cidx] = 0;
    }
  }
  const PassDesc pd = sc.pass[pass];
  const uint32_t n = sc.n;
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  if (!pd.active || tile >= ntiles) return;
  uint32_t* __restrict__ st = ctl->status[reg];
  const uint32_t base = tile * (uint32_t)kSortTile;
  const uint32_t cnt = min((uint32_t)kSortTile, n - base);
  const uint32_t shift = pd.shift;
  const uint64_t* __restrict__ in = pd.in;
  const int32_t* __restrict__ src = ctl->src;
  const int32_t* __restrict__ dst = ctl->dst;
  int32_t* cols = reinterpret_cast<int32_t*>(&S.keys[0]);  // first pass: src | dst

  // 0. bulk copy of the tile (what is not a multiple of 16 bytes, or not
  //    16-byte aligned, comes in with plain loads)
  uint32_t bulk;
  if (in) bulk = cnt & ~1u;
  else bulk = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0 ? (cnt & ~3u) : 0u;
  if (tid == 0) {
    const uint32_t bytes = bulk * 8u;  // 8-byte keys, or two 4-byte columns
    mbar_arrive_expect_tx(&S.bar, bytes);
    if (bulk) {
      if (in) {
        bulk_g2s(&S.keys[0], in + base, bulk * 8u, &S.bar);
      } else {
        bulk_g2s(cols, src + base, bulk * 4u, &S.bar);
        bulk_g2s(cols + kSortTile, dst + base, bulk * 4u, &S.bar);
      }
    }
    S.ok = mbar_wait_bounded(&S.bar, 0, &ctl->err) ? 1u : 0u;
  }
  if (in) {
    for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) S.keys[j] = in[base + j];
  } else {
    for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) {
      cols[j] = src[base + j];
      cols[kSortTile + j] = dst[base + j];
    }
  }
  __syncthreads();
  if (!S.ok) {  // the copy did not land in time (never expected)
    if (tid == 0) {
      atomicOr(&ctl->err, kErrLookback);
      mbar_wait_bounded(&S.bar, 0, nullptr);
    }
    return;
  }
  while (!mbar_try_wait(&S.bar, 0)) {
  }
  auto digit_at = [&](uint32_t j) -> uint32_t {
    if (in) return (uint32_t)(S.keys[j] >> shift) & (kRadix - 1);
    // packed key = bias(src) << 32 | bias(dst)
    const uint32_t v = shift >= 32 ? ((uint32_t)cols[j] ^ kBias) : ((uint32_t)cols[kSortTile + j] ^ kBias);
    return (v >> (shift & 31)) & (kRadix - 1);
  };
  const uint32_t wslot = warp * (kSortItems * 32);
  // 1. counts
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32 + lane;
    if (j < cnt) atomicAdd(&S.whist[warp][digit_at(j)], 1u);
  }
  __syncthreads();
  // 2. thread tid owns digit tid
  uint32_t bin_total = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = S.whist[w][tid];
    S.whist[w][tid] = bin_total;
    bin_total += c;
  }
  uint32_t* my_st = st + (size_t)tile * kRadix + tid;
  st_relaxed_u32(my_st, tile == 0 ? (kStInc | bin_total) : (1u + bin_total));
  const uint32_t chunk = tile >> kChunkShift;
  uint32_t* cagg = ctl->chunk_agg[reg];
  uint32_t* cinc = ctl->chunk_inc[reg];
  uint32_t* ccnt = ctl->chunk_cnt[reg];
  if (bin_total) atomicAdd(cagg + (size_t)chunk * kRadix + tid, bin_total);
  uint32_t tile_total;
  const uint32_t bin_start = block_exclusive_sum<kSortThreads>(bin_total, S.sw, tile_total);
  if (tid == 0) {
    // the block barrier inside the sum orders every thread's chunk-aggregate
    // add before this fence (fences are cumulative), so one release fence
    // makes all of them visible before the chunk counter moves
    __threadfence();
    atomicAdd(ccnt + chunk, 1u);
  }
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) S.whist[w][tid] += bin_start;
  __syncthreads();
  // 3. ranks
  const uint32_t lt = lanemask_lt();
  uint32_t* wmask = S.mask[warp];
  uint32_t* whist = S.whist[warp];
  uint32_t lpos[kSortItems / 2];  // two 16-bit positions per register
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32 + lane;
    const bool ok = j < cnt;
    const uint32_t dig = ok ? digit_at(j) : kRadix;
    atomicOr(&wmask[dig], 1u << lane);
    __syncwarp();
    const uint32_t peers = wmask[dig];
    __syncwarp();
    const int leader = 31 - __clz(peers);
    uint32_t old = 0;
    if (lane == leader) {
      wmask[dig] = 0;
      if (ok) old = atomicAdd(&whist[dig], (uint32_t)__popc(peers));
    }
    __syncwarp();
    old = __shfl_sync(0xFFFFFFFFu, old, leader);
    const uint32_t pos = old + __popc(peers & lt);
    if (i & 1) lpos[i >> 1] |= pos << 16;
    else lpos[i >> 1] = pos;
  }
  // 4. move the keys to their ranked places
  uint64_t key[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32 + lane;
    if (in) {
      key[i] = S.keys[j];
    } else {
      key[i] = ((uint64_t)((uint32_t)cols[j] ^ kBias) << 32) | ((uint32_t)cols[kSortTile + j] ^ kBias);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32 + lane;
    if (j < cnt) S.keys[(lpos[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu] = key[i];
  }
  // 5. look-back
  uint32_t excl = 0;
  if (tile > 0) {
    excl = digit_lookback2(st, cagg, cinc, ccnt, tile, ntiles, tid, ctl);
    st_relaxed_u32(my_st, kStInc | (excl + bin_total));
  }
  if ((tile & (kChunkTiles - 1)) == 0 && chunk > 0)
    st_relaxed_u32(cinc + (size_t)(chunk - 1) * kRadix + tid, kStInc | excl);
  if ((tile & (kChunkTiles - 1)) == kChunkTiles - 1 || tile == ntiles - 1)
    st_relaxed_u32(cinc + (size_t)chunk * kRadix + tid, kStInc | (excl + bin_total));
  S.delta[tid] = (int32_t)(sc.base[pass][tid] + excl) - (int32_t)bin_start;
  __syncthreads();
  // 6. scatter
  uint64_t* __restrict__ out = pd.out;
#pragma unroll 4
  for (uint32_t j = tid; j < cnt; j += kSortThreads) {
    const uint64_t k = S.keys[j];
    const uint32_t dig = (uint32_t)(k >> shift) & (kRadix - 1);
    const uint32_t pos = (uint32_t)(S.delta[dig] + (int32_t)j);
    if (pos < n) out[pos] = k;
  }
}

static std::mutex g_sweep_attr_mu;
static uint64_t g_sweep_attr_devs = 0;  // bit d: set on device d

// The onesweep kernel's dynamic shared memory limit, set once per device
// (not a stream operation, so it must happen before any stream capture).
void prepare_launches() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sweep_attr_mu);
  if (dev < 64 && !((g_sweep_attr_devs >> dev) & 1)) {
    cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SweepV6Smem));
    g_sweep_attr_devs |= 1ull << dev;
  }
}

void launch_onesweep(const Launch& L, int which, int pass, int gpass, uint32_t* counter,
                     cudaStream_t s) {
  if (L.row_slots == 0) return;
  prepare_launches();
  k_onesweep<<<L.row_slots, kSortThreads, sizeof(SweepV6Smem), s>>>(L.ctls, L.rows, counter,
                                                                    which, pass, gpass);
}

}  // namespace ringo
