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
    uint32_t* dst = &ctls[sidx].out_sort.hist[0];  // pass p, digit d at [p * 256 + d]
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
//   which = 0: out-sort of n_rows keys packed from the columns, 8-bit digits
//              at bits 0..63 (passes 0-3: dst, 4-7: src); between pass 3 and
//              pass 4 the dst-rank step always runs (it also packs from the
//              columns when every dst pass was skipped); buffers keysA/keysB.
//   which = 1: in-sort of E keys held in the out-sort's spare buffer, digits
//              of in_bits (8 or 9) bits from bit 32 up (the dst-run half).
__global__ void __launch_bounds__(kMaxRadix) k_plan(Ctl* __restrict__ ctls, int which, int in_bits) {
  Ctl* __restrict__ ctl = ctls + blockIdx.x;
  __shared__ uint32_t sw[kMaxRadix / 32 + 1];
  __shared__ uint32_t trivial[kOutPasses];
  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const int npass = which ? kInPasses : kOutPasses;
  const uint32_t n = which ? ctl->E : ctl->n_rows;
  const int rb = which ? in_bits : kRadixBits;
  const uint32_t R = 1u << rb;
  const uint32_t d = threadIdx.x;
  if (d < kOutPasses) trivial[d] = 0;
  __syncthreads();
  for (int p = 0; p < npass; ++p) {
    const uint32_t c = d < R ? sc.hist[(p << rb) + d] : 0u;
    uint32_t total;
    const uint32_t excl = block_exclusive_sum<kMaxRadix>(c, sw, total);
    if (d < R) {
      sc.base[(p << rb) + d] = excl;
      if (c == n) trivial[p] = 1;
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  sc.n = n;
  sc.bits = (uint32_t)rb;
  uint64_t* const b0 = which ? ctl->out_sort.spare : ctl->keysA;
  uint64_t* const b1 = which ? ctl->out_sort.result : ctl->keysB;
  const uint64_t* cur = which ? b0 : nullptr;
  uint64_t* next = which ? b1 : b0;
  uint32_t active = 0;
  const uint32_t shift0 = which ? 32 : 0;
  for (int p = 0; p < kOutPasses; ++p) {
    sc.pass[p].shift = p < npass ? shift0 + (uint32_t)rb * p : 0u;
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
  if (L.nseg) k_plan<<<L.nseg, kMaxRadix, 0, s>>>(L.ctls, which, L.opts.in_digit_bits == 9 ? 9 : 8);
}

// ---------------------------------------------------------------- K2/K4 ---
// One onesweep LSD pass: one block per tile of kSortTile keys, tiles claimed
// in increasing order through an atomic counter (the kernel and its per-tile
// steps are described at k_onesweep below).  which: 0 out-sort, 1 in-sort.
// pass: index within that sort.  gpass: global pass number; status region
// gpass&1 is used, and every processed tile clears its row of region
// (gpass+1)&1 for the next pass (the first `clear_words` words of the row:
// that pass's digit count).  A tile waits only on smaller tiles, every one
// of which was claimed by a block that is resident or done and never waits
// on a larger tile, so the waits always end.  Rows of both regions are
// kStRow words apart whatever the digit width.

// Two-level decoupled look-back for digit d of `tile`: first over the
// earlier tiles of the tile's own chunk (their aggregates or an inclusive
// prefix, kLbTiles status words per round trip), then over earlier chunks,
// kLbChunks per round trip: a chunk whose inclusive prefix is known ends the
// walk, a chunk whose tiles have all added their counts contributes its
// aggregate.  Every word read is self-validating (flag or tile count in the
// same word), so all loads are relaxed and a round needs no fence.  A
// chunk's aggregate is complete soon after its tiles have counted, so no
// wait follows the chain of inclusive prefixes tile by tile.  Bounded like
// every wait here.
constexpr int kLbTiles = kChunkTiles / 2;
constexpr int kLbChunks = 4;
__device__ __forceinline__ uint32_t digit_lookback2(const uint32_t* __restrict__ st,
                                                    const uint64_t* __restrict__ cagg,
                                                    const uint32_t* __restrict__ cinc,
                                                    uint32_t tile, uint32_t ntiles, uint32_t d,
                                                    Ctl* ctl) {
  const volatile uint32_t* verr = &ctl->err;
  uint32_t excl = 0, spins = 0;
  const uint32_t c = tile >> kChunkShift;
  const uint32_t first = c << kChunkShift;
  // 1. tiles [first, tile) of this chunk
  int64_t j = (int64_t)tile - 1;
  while (j >= (int64_t)first) {
    uint32_t v[kLbTiles];
#pragma unroll
    for (int k = 0; k < kLbTiles; ++k)
      v[k] = (j - k >= (int64_t)first) ? ld_relaxed_u32(st + (size_t)(j - k) * kStRow + d) : 0u;
    int used = 0;
    bool done = false, stall = false;
#pragma unroll
    for (int q = 0; q < kLbTiles; ++q) {
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
      if (spin_backoff(spins, ctl->spin_limit) || ((spins & 255) == 0 && *verr)) {
        atomicOr(&ctl->err, kErrLookback);
        return excl;
      }
    }
  }
  // 2. chunks c-1, c-2, ...
  int64_t cc = (int64_t)c - 1;
  while (cc >= 0) {
    uint32_t inc[kLbChunks];
    uint64_t agg[kLbChunks];
#pragma unroll
    for (int k = 0; k < kLbChunks; ++k) {
      const bool in = cc - k >= 0;
      inc[k] = in ? ld_relaxed_u32(cinc + (size_t)(cc - k) * kStRow + d) : 0u;
      agg[k] = in ? ld_relaxed_u64(cagg + (size_t)(cc - k) * kStRow + d) : 0ull;
    }
    int used = 0;
    bool done = false, stall = false;
#pragma unroll
    for (int k = 0; k < kLbChunks; ++k) {
      if (done || stall || cc - k < 0) continue;
      if (inc[k] & kStInc) {
        excl += inc[k] & ~kStInc;
        done = true;
        continue;
      }
      const uint32_t need =
          min((uint32_t)kChunkTiles, ntiles - ((uint32_t)(cc - k) << kChunkShift));
      if ((uint32_t)(agg[k] >> 32) >= need) {
        excl += (uint32_t)agg[k];
        used = k + 1;
      } else {
        stall = true;
      }
    }
    if (done) return excl;
    cc -= used;
    if (stall) {
      if (spin_backoff(spins, ctl->spin_limit) || ((spins & 255) == 0 && *verr)) {
        atomicOr(&ctl->err, kErrLookback);
        return excl;
      }
    }
  }
  return excl;
}

// The pass.  One 4096-key tile per block, three or four blocks per SM.  Per
// tile:
//   0. the tile arrives in shared memory by one bulk asynchronous copy
//      (cp.async.bulk + mbarrier; the first pass copies the two columns and
//      packs the keys as it reads them);
//   1. digit counts per warp (shared-memory adds), published at once, also
//      into the chunk aggregate of the two-level look-back;
//   2. thread t owns digits [t * DPT, t * DPT + DPT), DPT = digits / 256:
//      per-warp starts within the tile;
//   3. stable ranks: the lanes of a warp holding the same digit find each
//      other (through a shared lane mask, one ballot per digit bit, or a
//      warp match); the highest of them advances the warp's running position
//      of that digit for the whole group, so each key gets its final place
//      in the staged tile;
//   4. the keys move to their places in the same buffer;
//   5. two-level look-back (thread t, its digits) -> global digit offsets;
//   6. coalesced scatter of the staged tile.
// An 8-bit digit is byte BYTE of the key's high or low word (a template
// parameter, taken with one byte permute); a 9-bit digit is taken with a
// shift and a mask.  Full tiles take a path without bounds checks, so the
// per-key work is a few shared-memory operations and no branches.

// What thread 0 learns about the block's tile, for the whole block.
struct SweepTile {
  uint32_t valid;  // 0: no slot left
  uint32_t work;   // 1: this pass moves keys of this tile
  uint32_t seg, tile, slot;
  uint32_t n;      // keys of this sort in the tile's segment
  uint32_t cnt;    // keys in the tile
  uint32_t bulk;   // keys brought by the bulk copy; the rest by plain loads
  uint32_t shift;  // position of the digit within its 32-bit word
  const uint64_t* in;  // NULL: pack from the columns
  uint64_t* out;
};

template <int R, int RANK>
struct SweepSmem {
  uint64_t keys[kSortTile];       // the tile: input, then staged in digit order
  uint32_t whist[kSortWarps][R];  // per-warp counts, then running positions
  // peer masks (lane-mask ranking only); slot R: lanes past the end
  uint32_t mask[RANK == 0 ? kSortWarps : 1][RANK == 0 ? R + 1 : 1];
  uint32_t delta[R];              // global place of a staged key minus its index
  uint32_t sw[kSortWarps + 1];
  SweepTile t;
  uint64_t bar;
};

__host__ __device__ constexpr size_t sweep_smem_bytes(int bits, int rank) {
  return bits > 8 ? (rank == 0 ? sizeof(SweepSmem<512, 0>) : sizeof(SweepSmem<512, 1>))
                  : (rank == 0 ? sizeof(SweepSmem<256, 0>) : sizeof(SweepSmem<256, 1>));
}

template <int RB, int BYTE>
__device__ __forceinline__ uint32_t digit_of(uint32_t w, uint32_t sh) {
  if constexpr (BYTE >= 0) {
    return __byte_perm(w, 0u, 0x4440u + BYTE);
  } else {
    return (w >> sh) & ((1u << RB) - 1u);
  }
}

// The word of key j that holds this pass's digit.  Packed first pass: the
// columns sit in the tile buffer as src[0..4096) then dst[0..4096).
template <bool HI, bool PACK, class SM>
__device__ __forceinline__ uint32_t key_word(const SM& S, uint32_t j) {
  if (PACK) {
    const int32_t* cols = reinterpret_cast<const int32_t*>(S.keys);
    return (uint32_t)cols[HI ? j : kSortTile + j] ^ kBias;
  }
  const uint64_t k = S.keys[j];
  return HI ? (uint32_t)(k >> 32) : (uint32_t)k;
}
template <bool PACK, class SM>
__device__ __forceinline__ uint64_t key_at(const SM& S, uint32_t j) {
  if (PACK) {
    const int32_t* cols = reinterpret_cast<const int32_t*>(S.keys);
    return ((uint64_t)((uint32_t)cols[j] ^ kBias) << 32) | ((uint32_t)cols[kSortTile + j] ^ kBias);
  }
  return S.keys[j];
}

// Steps 1-6 for one tile of `cnt` keys (FULL: cnt == kSortTile); `sh` is the
// digit's position within its word (9-bit digits).
template <int RB, int BYTE, bool HI, int RANK, bool PACK, bool FULL>
__device__ __forceinline__ void sweep_body(SweepSmem<(1 << RB), RANK>& S, Ctl* __restrict__ ctl,
                                           SortCtl& sc, uint64_t* __restrict__ out, uint32_t tile,
                                           uint32_t ntiles, uint32_t cnt, uint32_t n, int pass,
                                           int reg, uint32_t sh) {
  constexpr int R = 1 << RB;
  constexpr int DPT = R / kSortThreads;
  static_assert(DPT == 1 || DPT == 2, "one or two digits per thread");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t wslot = warp * (kSortItems * 32) + lane;
  const uint32_t d0 = (uint32_t)tid * DPT;  // this thread's first digit
  // 1. counts
  uint32_t* whist = S.whist[warp];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32;
    if (FULL || j < cnt) atomicAdd(whist + digit_of<RB, BYTE>(key_word<HI, PACK>(S, j), sh), 1u);
  }
  __syncthreads();
  // 2. thread tid owns digits d0 .. d0 + DPT - 1
  uint32_t c[DPT][kSortWarps];
  uint32_t bin_total[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) bin_total[k] = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    if constexpr (DPT == 1) {
      c[0][w] = S.whist[w][tid];
    } else {
      const uint2 v = reinterpret_cast<const uint2*>(S.whist[w])[tid];
      c[0][w] = v.x;
      c[DPT - 1][w] = v.y;
    }
#pragma unroll
    for (int k = 0; k < DPT; ++k) bin_total[k] += c[k][w];
  }
  uint32_t* __restrict__ st = ctl->status[reg];
  uint32_t* my_st = st + (size_t)tile * kStRow + d0;
  const uint32_t chunk = tile >> kChunkShift;
  uint64_t* cagg = ctl->chunk_agg[reg];
  uint32_t* cinc = ctl->chunk_inc[reg];
  uint32_t my_total = 0;
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    st_relaxed_u32(my_st + k, tile == 0 ? (kStInc | bin_total[k]) : (1u + bin_total[k]));
    // one more tile of this chunk, and its count, in one atomic word
    atomicAdd(reinterpret_cast<unsigned long long*>(cagg + (size_t)chunk * kStRow + d0 + k),
              (1ull << 32) | bin_total[k]);
    my_total += bin_total[k];
  }
  uint32_t tile_total;
  const uint32_t start0 = block_exclusive_sum<kSortThreads>(my_total, S.sw, tile_total);
  uint32_t bin_start[DPT];
  {
    uint32_t run = start0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      bin_start[k] = run;
      run += bin_total[k];
    }
  }
  {
    uint32_t run[DPT];
#pragma unroll
    for (int k = 0; k < DPT; ++k) run[k] = bin_start[k];
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      if constexpr (DPT == 1) {
        S.whist[w][tid] = run[0];
      } else {
        reinterpret_cast<uint2*>(S.whist[w])[tid] = make_uint2(run[0], run[DPT - 1]);
      }
#pragma unroll
      for (int k = 0; k < DPT; ++k) run[k] += c[k][w];
    }
  }
  __syncthreads();
  // 3. ranks -> places in the staged tile
  const uint32_t lt = lanemask_lt();
  const uint32_t bit = 1u << lane;
  const uint32_t wmask = RANK == 0 ? smem_addr(S.mask[warp]) : 0u;
  const uint32_t whaddr = smem_addr(whist);
  uint32_t lpos[kSortItems / 2];  // two 16-bit places per register
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t j = wslot + i * 32;
    const bool ok = FULL || j < cnt;
    const uint32_t d = ok ? digit_of<RB, BYTE>(key_word<HI, PACK>(S, j), sh) : (uint32_t)R;
    uint32_t peers, old = 0;
    if constexpr (RANK == 0) {
      asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(wmask + 4 * d), "r"(bit) : "memory");
      __syncwarp();
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(peers) : "r"(wmask + 4 * d) : "memory");
      __syncwarp();
    } else if constexpr (RANK == 1) {
      // one ballot per digit bit (and one for "past the end" in a partial
      // tile): the lanes that agree on every bit
      peers = 0xFFFFFFFFu;
#pragma unroll
      for (int q = 0; q < (FULL ? RB : RB + 1); ++q) {
        const bool b = (d >> q) & 1u;
        const uint32_t bb = __ballot_sync(0xFFFFFFFFu, b);
        peers &= b ? bb : ~bb;
      }
    } else {
      peers = __match_any_sync(0xFFFFFFFFu, d);
    }
    const uint32_t leader = 31u - __clz(peers);
    // the group's highest lane (clears the mask entry and) advances the
    // digit's running place by the group size (predicated, no branch)
    const uint32_t lead = ((uint32_t)lane == leader) & (ok ? 1u : 0u);
    if constexpr (RANK == 0) {
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
          " @p st.shared.u32 [%2], 0;\n"
          " @p atom.shared.add.u32 %0, [%3], %4;\n}\n"
          : "+r"(old)
          : "r"(lead), "r"(wmask + 4 * d), "r"(whaddr + 4 * d), "r"((uint32_t)__popc(peers))
          : "memory");
    } else {
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
          " @p atom.shared.add.u32 %0, [%2], %3;\n}\n"
          : "+r"(old)
          : "r"(lead), "r"(whaddr + 4 * d), "r"((uint32_t)__popc(peers))
          : "memory");
    }
    __syncwarp();
    old = __shfl_sync(0xFFFFFFFFu, old, leader);
    const uint32_t pos = old + (uint32_t)__popc(peers & lt);
    if (i & 1) lpos[i >> 1] |= pos << 16;
    else lpos[i >> 1] = pos;
  }
  // 4. keys to their places
  uint64_t key[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) key[i] = key_at<PACK>(S, wslot + i * 32);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (FULL || wslot + i * 32 < cnt) S.keys[(lpos[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu] = key[i];
  }
  // 5. look-back, one walk per digit; each digit's inclusive prefix is
  // published as soon as it is known
  uint32_t excl[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    excl[k] = 0;
    if (tile > 0) {
      excl[k] = digit_lookback2(st, cagg, cinc, tile, ntiles, d0 + k, ctl);
      st_relaxed_u32(my_st + k, kStInc | (excl[k] + bin_total[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    if ((tile & (kChunkTiles - 1)) == 0 && chunk > 0)
      st_relaxed_u32(cinc + (size_t)(chunk - 1) * kStRow + d0 + k, kStInc | excl[k]);
    if ((tile & (kChunkTiles - 1)) == kChunkTiles - 1 || tile == ntiles - 1)
      st_relaxed_u32(cinc + (size_t)chunk * kStRow + d0 + k, kStInc | (excl[k] + bin_total[k]));
    // modulo 2^32: the sum below is the key's place, which is below n
    S.delta[d0 + k] = sc.base[(pass << RB) + d0 + k] + excl[k] - bin_start[k];
  }
  __syncthreads();
  // 6. scatter
#pragma unroll
  for (int q = 0; q < kSortItems; ++q) {
    const uint32_t j = (uint32_t)tid + q * kSortThreads;
    if (FULL || j < cnt) {
      const uint64_t k = S.keys[j];
      const uint32_t w = HI ? (uint32_t)(k >> 32) : (uint32_t)k;
      const uint32_t pos = S.delta[digit_of<RB, BYTE>(w, sh)] + j;
      if (pos < n) out[pos] = k;
    }
  }
}

template <int RB, int BYTE, bool HI, int RANK>
__global__ void __launch_bounds__(kSortThreads, sweep_blocks_per_sm(RB, RANK))
    k_onesweep(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter, int which, int pass,
               int gpass, uint32_t ahead_slots, uint32_t clear_words) {
  constexpr int R = 1 << RB;
  using Smem = SweepSmem<R, RANK>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&S.bar, 1);
    mbar_init_fence();
    const uint32_t g = atomicAdd(counter, 1u);
    const uint32_t total = __ldg(m.start + m.nseg);
    // the first segment's fields are read while the claim is in flight: a
    // single-table launch needs nothing else before its copy starts
    const Ctl* c = ctls;
    const SortCtl* sc = which ? &c->in_sort : &c->out_sort;
    PassDesc pd = sc->pass[pass];
    uint32_t n = sc->n;
    SweepTile t{};
    t.slot = g;
    if (g < total) {
      uint32_t seg = 0, tile = g;
      if (m.nseg > 1) {
        seg = seg_of(m, g);
        tile = g - __ldg(m.start + seg);
        c = ctls + seg;
        sc = which ? &c->in_sort : &c->out_sort;
        pd = sc->pass[pass];
        n = sc->n;
      }
      t.valid = 1;
      t.seg = seg;
      t.tile = tile;
      t.n = n;
      t.shift = pd.shift & 31u;
      if (pd.active && tile < (n + kSortTile - 1) / kSortTile) {
        const uint32_t base = tile * (uint32_t)kSortTile;
        t.work = 1;
        t.cnt = min((uint32_t)kSortTile, n - base);
        t.in = pd.in;
        t.out = pd.out;
        // bulk copy of the tile (what is not a multiple of 16 bytes, or not
        // 16-byte aligned, comes in with plain loads)
        if (pd.in) {
          t.bulk = t.cnt & ~1u;
          mbar_arrive_expect_tx(&S.bar, t.bulk * 8u);
          if (t.bulk) bulk_g2s(&S.keys[0], pd.in + base, t.bulk * 8u, &S.bar);
        } else {
          const int32_t* src = c->src;
          const int32_t* dst = c->dst;
          t.bulk = ((((uintptr_t)src) | ((uintptr_t)dst)) & 15) == 0 ? (t.cnt & ~3u) : 0u;
          mbar_arrive_expect_tx(&S.bar, t.bulk * 8u);  // two 4-byte columns
          if (t.bulk) {
            int32_t* cols = reinterpret_cast<int32_t*>(&S.keys[0]);
            bulk_g2s(cols, src + base, t.bulk * 4u, &S.bar);
            bulk_g2s(cols + kSortTile, dst + base, t.bulk * 4u, &S.bar);
          }
        }
      }
    }
    S.t = t;
    // the tile a block will claim `ahead_slots` claims from now (a whole
    // number of waves of resident blocks) goes to L2 already, so that
    // block's copy does not wait on DRAM
    const uint32_t ahead = g + ahead_slots;
    if (ahead_slots && ahead < total) {
      const uint32_t ps = m.nseg > 1 ? seg_of(m, ahead) : 0u;
      const uint32_t pt = ahead - (m.nseg > 1 ? __ldg(m.start + ps) : 0u);
      const Ctl* pc = ctls + ps;
      const SortCtl& psc = which ? pc->in_sort : pc->out_sort;
      const uint32_t pn = psc.n, pb = pt * (uint32_t)kSortTile;
      if (psc.pass[pass].active && pb < pn) {
        const uint32_t pcnt = min((uint32_t)kSortTile, pn - pb);
        const uint64_t* pin = psc.pass[pass].in;
        if (pin) {
          if (pcnt & ~1u) bulk_prefetch_l2(pin + pb, (pcnt & ~1u) * 8u);
        } else if (((((uintptr_t)pc->src) | ((uintptr_t)pc->dst)) & 15) == 0 && (pcnt & ~3u)) {
          bulk_prefetch_l2(pc->src + pb, (pcnt & ~3u) * 4u);
          bulk_prefetch_l2(pc->dst + pb, (pcnt & ~3u) * 4u);
        }
      }
    }
  }
  for (int i = tid; i < kSortWarps * R; i += kSortThreads) (&S.whist[0][0])[i] = 0;
  if constexpr (RANK == 0) {
    for (int i = tid; i < kSortWarps * (R + 1); i += kSortThreads) (&S.mask[0][0])[i] = 0;
  }
  __syncthreads();
  const SweepTile t = S.t;
  if (!t.valid) return;
  Ctl* __restrict__ ctl = ctls + t.seg;
  const uint32_t tile = t.tile;
  const int reg = gpass & 1, nreg = reg ^ 1;
  if (tile < ctl->status_rows) {
    // clear this tile's row (and, for a chunk's first tile, the chunk's row)
    // of the other region for the next pass
    uint32_t* row = ctl->status[nreg] + (size_t)tile * kStRow;
    for (uint32_t i = tid; i < clear_words; i += kSortThreads) row[i] = 0;
    if ((tile & (kChunkTiles - 1)) == 0) {
      const size_t cbase = (size_t)(tile >> kChunkShift) * kStRow;
      for (uint32_t i = tid; i < clear_words; i += kSortThreads) {
        ctl->chunk_agg[nreg][cbase + i] = 0;
        ctl->chunk_inc[nreg][cbase + i] = 0;
      }
    }
  }
  if (!t.work) return;
  const uint32_t n = t.n, cnt = t.cnt, bulk = t.bulk;
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  const uint32_t base = tile * (uint32_t)kSortTile;
  if (cnt > bulk) {
    if (t.in) {
      for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) S.keys[j] = t.in[base + j];
    } else {
      int32_t* cols = reinterpret_cast<int32_t*>(&S.keys[0]);
      for (uint32_t j = bulk + tid; j < cnt; j += kSortThreads) {
        cols[j] = ctl->src[base + j];
        cols[kSortTile + j] = ctl->dst[base + j];
      }
    }
  }
  // every thread waits for the copy; the block agrees before going on
  const bool ok = mbar_wait_bounded(&S.bar, 0, &ctl->err, ctl->spin_limit);
  if (!__syncthreads_and(ok)) {  // the copy did not land in time (never expected)
    if (tid == 0) {
      atomicOr(&ctl->err, kErrLookback);
      mbar_wait_bounded(&S.bar, 0, nullptr);
    }
    return;
  }
  SortCtl& sc = which ? ctl->in_sort : ctl->out_sort;
  const bool full = cnt == (uint32_t)kSortTile;
  const uint32_t sh = t.shift;
  if constexpr (!HI) {
    if (!t.in) {
      if (full) sweep_body<RB, BYTE, HI, RANK, true, true>(S, ctl, sc, t.out, tile, ntiles, cnt, n, pass, reg, sh);
      else sweep_body<RB, BYTE, HI, RANK, true, false>(S, ctl, sc, t.out, tile, ntiles, cnt, n, pass, reg, sh);
      return;
    }
  }
  if (full) sweep_body<RB, BYTE, HI, RANK, false, true>(S, ctl, sc, t.out, tile, ntiles, cnt, n, pass, reg, sh);
  else sweep_body<RB, BYTE, HI, RANK, false, false>(S, ctl, sc, t.out, tile, ntiles, cnt, n, pass, reg, sh);
}

using SweepFn = void (*)(Ctl*, SegMap, uint32_t*, int, int, int, uint32_t, uint32_t);
// 8-bit digits, [rank method][hi][byte]: the digit of out-sort pass p is
// byte p % 4 of the low word (p < 4) or of the high word; in-sort pass p is
// byte p of the high word.  9-bit digits (in-sort only), [rank method]: bits
// 9p .. 9p+8 of the high word.
#define RINGO_SWEEPS8(R)                                                                     \
  {{k_onesweep<8, 0, false, R>, k_onesweep<8, 1, false, R>, k_onesweep<8, 2, false, R>,     \
    k_onesweep<8, 3, false, R>},                                                             \
   {k_onesweep<8, 0, true, R>, k_onesweep<8, 1, true, R>, k_onesweep<8, 2, true, R>,        \
    k_onesweep<8, 3, true, R>}}
static const SweepFn kSweep8[3][2][4] = {RINGO_SWEEPS8(0), RINGO_SWEEPS8(1), RINGO_SWEEPS8(2)};
#undef RINGO_SWEEPS8
static const SweepFn kSweep9[3] = {k_onesweep<9, -1, true, 0>, k_onesweep<9, -1, true, 1>,
                                   k_onesweep<9, -1, true, 2>};

static std::mutex g_sweep_attr_mu;
static uint64_t g_sweep_attr_devs = 0;  // bit d: set on device d

// The onesweep kernels' dynamic shared memory limit, set once per device
// (not a stream operation, so it must happen before any stream capture).
void prepare_launches() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sweep_attr_mu);
  if (dev < 64 && !((g_sweep_attr_devs >> dev) & 1)) {
    for (int r = 0; r < 3; ++r) {
      for (int h = 0; h < 2; ++h)
        for (int b = 0; b < 4; ++b)
          cudaFuncSetAttribute(kSweep8[r][h][b], cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sweep_smem_bytes(8, r));
      cudaFuncSetAttribute(kSweep9[r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sweep_smem_bytes(9, r));
    }
    g_sweep_attr_devs |= 1ull << dev;
  }
}

void launch_onesweep(const Launch& L, int which, int pass, int gpass, uint32_t* counter,
                     cudaStream_t s) {
  if (L.row_slots == 0) return;
  prepare_launches();
  const int rank = L.opts.rank_method >= 0 && L.opts.rank_method <= 2 ? L.opts.rank_method : 0;
  const int in_bits = L.opts.in_digit_bits == 9 ? 9 : 8;
  const int bits = which ? in_bits : kRadixBits;
  SweepFn fn;
  if (bits == 9) {
    fn = kSweep9[rank];
  } else {
    // shift = (which ? 32 : 0) + 8 * pass; see k_plan
    const int shift = (which ? 32 : 0) + kRadixBits * pass;
    fn = kSweep8[rank][shift >= 32][(shift & 31) >> 3];
  }
  // the digit count of the pass that uses the other status region next
  const uint32_t clear = gpass + 1 < kOutPasses ? (uint32_t)kRadix : (1u << in_bits);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t waves = (uint32_t)max(0, min(2, L.opts.prefetch_waves));
  const uint32_t ahead = waves * sweep_blocks_per_sm(bits, rank) * (uint32_t)sms;
  fn<<<L.row_slots, kSortThreads, sweep_smem_bytes(bits, rank), s>>>(
      L.ctls, L.rows, counter, which, pass, gpass, ahead, clear);
}

}  // namespace ringo
