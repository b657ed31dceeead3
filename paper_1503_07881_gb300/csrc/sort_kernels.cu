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
//              bits 0..63; buffers keysA, keysB.
//   which = 1: in-sort of E keys held in the out-sort's spare buffer,
//              digits at bits 32..63 (the dst half).
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
    const bool last_chance = (p == npass - 1) && active == 0;
    if (trivial[p] && !last_chance) continue;
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
// One onesweep LSD pass over a tile of kSortTile keys.
//   which: 0 out-sort, 1 in-sort.   pass: pass index within that sort.
//   gpass: global pass number; status region gpass&1 is used, and this pass
//          clears its tile's row of region (gpass+1)&1 for the next pass.
// Tiles are numbered in the order blocks start (an atomic counter), so every
// tile a block waits on belongs to a block that is already running.
__global__ void __launch_bounds__(kSortThreads, 3)
    k_onesweep(Ctl* __restrict__ ctl, int which, int pass, int gpass) {
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

  // load: warp-striped, item i of lane l sits at wbase + 32 i + l
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

  // rank within the warp, in position order: peers with the same digit in
  // this item are found with match.any; the highest peer bumps the warp's
  // digit counter for the whole group.
  uint16_t rank[kSortItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const bool ok = (valid >> i) & 1u;
    const uint32_t dig = ok ? (uint32_t)(key[i] >> shift) & (kRadix - 1) : kRadix;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig);
    const int leader = 31 - __clz(peers);
    uint32_t old = 0;
    if (lane == leader && ok) old = atomicAdd(&s_whist[warp][dig], (uint32_t)__popc(peers));
    old = __shfl_sync(0xFFFFFFFFu, old, leader);
    rank[i] = (uint16_t)(old + __popc(peers & lt));
  }
  __syncthreads();

  // thread tid owns digit tid: prefix over warps, then the tile's digit count
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

  // decoupled look-back over earlier tiles for this digit
  uint32_t excl = 0;
  if (tile > 0) {
    uint32_t j = tile - 1;
    uint32_t spins = 0;
    while (true) {
      const uint32_t s = ld_relaxed_u32(st + (size_t)j * kRadix + tid);
      if (s == 0) {
        if (spin_backoff(spins)) {
          atomicOr(&ctl->err, kErrLookback);
          break;
        }
        continue;
      }
      if (s & kStInc) {
        excl += s & ~kStInc;
        break;
      }
      excl += s - 1u;
      if (j == 0) break;  // unreachable: tile 0 always publishes inclusive
      --j;
    }
    st_relaxed_u32(my_st, kStInc | (excl + bin_total));
  }
  s_delta[tid] = (int32_t)(sc.base[pass][tid] + excl) - (int32_t)bin_start;
  __syncthreads();

  // stage the tile in digit order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if ((valid >> i) & 1u) {
      const uint32_t dig = (uint32_t)(key[i] >> shift) & (kRadix - 1);
      s_keys[s_binstart[dig] + s_whist[warp][dig] + rank[i]] = key[i];
    }
  }
  __syncthreads();

  // coalesced scatter: consecutive staged keys of a digit go to consecutive
  // global positions
  const uint32_t nvalid = min((uint32_t)kSortTile, n - base);
  uint64_t* __restrict__ out = pd.out;
#pragma unroll 4
  for (uint32_t j = tid; j < nvalid; j += kSortThreads) {
    const uint64_t k = s_keys[j];
    const uint32_t dig = (uint32_t)(k >> shift) & (kRadix - 1);
    out[(uint32_t)(s_delta[dig] + (int32_t)j)] = k;
  }
}

void launch_onesweep(Ctl* ctl, int which, int pass, int gpass, uint32_t grid, cudaStream_t s) {
  if (grid == 0) return;
  k_onesweep<<<grid, kSortThreads, 0, s>>>(ctl, which, pass, gpass);
}

}  // namespace ringo
