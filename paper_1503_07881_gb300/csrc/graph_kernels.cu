// Kernels around the sorts: destination ranks between the dst and src
// passes, adjacent-duplicate removal with source-run extraction,
// destination-run starts after the in-sort, the node-list merge, the run
// index -> node index remap, and degree queries.
//
// These are the "computing the number of neighbors for each node, and then
// copying the neighbor vectors" steps of the paper's sort-first conversion
// (Section 3.4), done with single-pass compactions (decoupled look-back) so
// that every neighbour array is written once, in order, with no atomics on
// the data.
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"
#include "ringo_internal.cuh"

namespace ringo {

namespace {
constexpr int kWarps = kScanThreads / 32;

__device__ __forceinline__ int32_t unbias(uint32_t b) { return (int32_t)(b ^ kBias); }
__device__ __forceinline__ ScanChunks chunks_of(const Ctl* ctl, int i) {
  return ScanChunks{ctl->scan_chunk_agg[i], ctl->scan_chunk_inc[i], ctl->scan_chunk_cnt[i]};
}
}  // namespace

// ------------------------------------------------------------------ K3 ----
// Input: the out-sorted keys (bias(src) << 32 | dst-run index), n_rows of
// them.  A key that differs from its predecessor is a distinct edge e; a key
// whose src differs is the start of a source run s.  Outputs:
//   in-sort keys  spare[e]   = dst-run index << 32 | s_index(src)
//   out_nbr[e]               = dst-run index (turned into a node index later)
//   usrc[s], usrc_start[s]   = src ID and its first edge; usrc_start[Vs] = E
//   in_sort.hist             = digit histograms of the in-sort passes
__global__ void __launch_bounds__(kScanThreads)
    k_dedup(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ uint32_t s_hist[kInPasses][kRadix];
  __shared__ uint32_t s_we[kWarps], s_ws[kWarps];
  __shared__ uint64_t s_prefix;
  __shared__ Claim s_cl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) claim_slot(m, counter, &s_cl);
  for (int i = tid; i < kInPasses * kRadix; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t tile = s_cl.tile;
  const uint32_t n = ctl->n_rows;
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (tile >= ntiles) return;
  const uint64_t* __restrict__ keys = ctl->out_sort.result;
  const uint32_t wbase = tile * (uint32_t)kScanTile + warp * (kScanItems * 32);

  uint64_t key[kScanItems];
  uint32_t valid = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t pos = wbase + i * 32 + lane;
    key[i] = pos < n ? __ldcs(keys + pos) : 0;
    if (pos < n) valid |= 1u << i;
  }
  uint64_t before = 0;  // key just before this warp's first item
  if (wbase > 0 && wbase <= n) before = keys[wbase - 1];

  const uint32_t lt = lanemask_lt();
  uint32_t he = 0, hs = 0, ce = 0, cs = 0;
  uint16_t eloc[kScanItems], sloc[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, key[i], 1);
    const uint64_t last_prev_item = __shfl_sync(0xFFFFFFFFu, i ? key[i - 1] : before, 31);
    if (lane == 0) prev = i ? last_prev_item : before;
    const uint32_t pos = wbase + i * 32 + lane;
    const bool ok = (valid >> i) & 1u;
    const bool first = pos == 0;
    const bool h_e = ok && (first || key[i] != prev);
    const bool h_s = ok && (first || (key[i] >> 32) != (prev >> 32));
    const uint32_t be = __ballot_sync(0xFFFFFFFFu, h_e);
    const uint32_t bs = __ballot_sync(0xFFFFFFFFu, h_s);
    eloc[i] = (uint16_t)(ce + __popc(be & lt));
    sloc[i] = (uint16_t)(cs + __popc(bs & lt));
    ce += __popc(be);
    cs += __popc(bs);
    he |= (uint32_t)h_e << i;
    hs |= (uint32_t)h_s << i;
  }
  if (lane == 0) {
    s_we[warp] = ce;
    s_ws[warp] = cs;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t e = lane < kWarps ? s_we[lane] : 0;
    const uint32_t s = lane < kWarps ? s_ws[lane] : 0;
    const uint32_t ei = warp_inclusive_sum(e), si = warp_inclusive_sum(s);
    const uint32_t te = __shfl_sync(0xFFFFFFFFu, ei, 31), ts = __shfl_sync(0xFFFFFFFFu, si, 31);
    const uint64_t excl = scan_prefix(ctl->scan_status[0], chunks_of(ctl, 0), tile, ntiles,
                                      pack2(te, ts), &ctl->err);
    __syncwarp();
    if (lane < kWarps) {
      s_we[lane] = ei - e;
      s_ws[lane] = si - s;
    }
    if (lane == 0) {
      s_prefix = excl;
      if (tile == ntiles - 1) {
        const uint32_t E = unpackA(excl) + te, Vs = unpackB(excl) + ts;
        ctl->E = E;
        ctl->Vs = Vs;
        ctl->usrc_start[Vs] = (int32_t)E;
      }
    }
  }
  __syncthreads();
  const uint32_t e0 = unpackA(s_prefix) + s_we[warp];
  const uint32_t s0 = unpackB(s_prefix) + s_ws[warp];
  uint64_t* __restrict__ ekeys = ctl->out_sort.spare;
  int32_t* __restrict__ out_nbr = ctl->out_nbr;
  int32_t* __restrict__ usrc = ctl->usrc;
  int32_t* __restrict__ usrc_start = ctl->usrc_start;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (!((he >> i) & 1u)) continue;
    const uint32_t e = e0 + eloc[i];
    const uint32_t s = s0 + sloc[i];
    const bool head_s = (hs >> i) & 1u;
    const uint32_t sidx = head_s ? s : s - 1;
    const uint32_t db = (uint32_t)key[i];
    ekeys[e] = ((uint64_t)db << 32) | sidx;
    out_nbr[e] = (int32_t)db;
    atomicAdd(&s_hist[0][db & 0xFF], 1u);
    atomicAdd(&s_hist[1][(db >> 8) & 0xFF], 1u);
    atomicAdd(&s_hist[2][(db >> 16) & 0xFF], 1u);
    atomicAdd(&s_hist[3][db >> 24], 1u);
    if (head_s) {
      usrc[s] = unbias((uint32_t)(key[i] >> 32));
      usrc_start[s] = (int32_t)e;
    }
  }
  __syncthreads();
  for (int i = tid; i < kInPasses * kRadix; i += kScanThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(&ctl->in_sort.hist[0][0] + i, c);
  }
}

void launch_dedup(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (L.row_slots) k_dedup<<<L.row_slots, kScanThreads, 0, s>>>(L.ctls, L.rows, counter);
}

// ------------------------------------------------------------- dst rank ---
// Runs between out-sort passes 3 and 4, when the keys are in dst order.
// Each key's dst is replaced by its destination-run index (the rank of the
// dst among the distinct dst values), which keeps the key order; the run
// heads give udst[], the distinct destination IDs in ascending order.
// Reads rank_step.in (or packs from the columns when every dst pass was
// trivial) and writes rank_step.out.  Single-pass compaction count with
// decoupled look-back.
__global__ void __launch_bounds__(kScanThreads)
    k_dst_rank(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ uint32_t s_w[kWarps];
  __shared__ uint64_t s_prefix;
  __shared__ Claim s_cl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t tile = s_cl.tile;
  const uint32_t n = ctl->n_rows;
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (tile >= ntiles) return;
  const uint64_t* __restrict__ in = ctl->rank_step.in;
  uint64_t* __restrict__ out = ctl->rank_step.out;
  const int32_t* __restrict__ src = ctl->src;
  const int32_t* __restrict__ dst = ctl->dst;
  auto key_at = [&](uint32_t pos) -> uint64_t {
    if (in) return in[pos];
    return ((uint64_t)((uint32_t)src[pos] ^ kBias) << 32) | ((uint32_t)dst[pos] ^ kBias);
  };
  const uint32_t wbase = tile * (uint32_t)kScanTile + warp * (kScanItems * 32);
  uint64_t key[kScanItems];
  uint32_t valid = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t pos = wbase + i * 32 + lane;
    if (pos < n) {
      key[i] = in ? __ldcs(in + pos) : key_at(pos);
      valid |= 1u << i;
    } else {
      key[i] = 0;
    }
  }
  uint64_t before = 0;
  if (wbase > 0 && wbase <= n) before = key_at(wbase - 1);
  const uint32_t lt = lanemask_lt();
  uint32_t hd = 0, cd = 0;
  uint16_t dloc[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, key[i], 1);
    const uint64_t last_prev_item = __shfl_sync(0xFFFFFFFFu, i ? key[i - 1] : before, 31);
    if (lane == 0) prev = i ? last_prev_item : before;
    const uint32_t pos = wbase + i * 32 + lane;
    const bool ok = (valid >> i) & 1u;
    const bool h = ok && (pos == 0 || (uint32_t)key[i] != (uint32_t)prev);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
    dloc[i] = (uint16_t)(cd + __popc(b & lt));
    cd += __popc(b);
    hd |= (uint32_t)h << i;
  }
  if (lane == 0) s_w[warp] = cd;
  __syncthreads();
  if (warp == 0) {
    const uint32_t c = lane < kWarps ? s_w[lane] : 0;
    const uint32_t ci = warp_inclusive_sum(c);
    const uint32_t tc = __shfl_sync(0xFFFFFFFFu, ci, 31);
    const uint64_t excl = scan_prefix(ctl->scan_status[1], chunks_of(ctl, 1), tile, ntiles,
                                      pack2(0, tc), &ctl->err);
    __syncwarp();
    if (lane < kWarps) s_w[lane] = ci - c;
    if (lane == 0) {
      s_prefix = excl;
      if (tile == ntiles - 1) ctl->Vd = unpackB(excl) + tc;
    }
  }
  __syncthreads();
  const uint32_t d0 = unpackB(s_prefix) + s_w[warp];
  int32_t* __restrict__ udst = ctl->udst;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (!((valid >> i) & 1u)) continue;
    const bool h = (hd >> i) & 1u;
    const uint32_t r = d0 + dloc[i] + (h ? 0u : 0xFFFFFFFFu);  // inclusive count - 1
    __stcs(out + wbase + i * 32 + lane, (key[i] & 0xFFFFFFFF00000000ull) | r);
    if (h) udst[r] = unbias((uint32_t)key[i]);
  }
}

void launch_dst_rank(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (L.row_slots) k_dst_rank<<<L.row_slots, kScanThreads, 0, s>>>(L.ctls, L.rows, counter);
}

// ------------------------------------------------------------------ K5 ----
// Input: the in-sorted keys (dst-run index << 32 | source-run index), E of
// them, in (dst, src) order.  Writes in_nbr[k] = source-run index (turned
// into a node index later) and, at each change of dst-run index d, the run's
// first in-edge udst_start[d] = k (udst_start[Vd] = E).  Every dst-run index
// occurs, so no compaction is needed.
__global__ void __launch_bounds__(256)
    k_dst_runs(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t E = ctl->E, Vd = ctl->Vd;
  const uint32_t base = s_cl.tile * (uint32_t)kScanTile;
  if (base >= E) return;
  const uint32_t end = min(E, base + (uint32_t)kScanTile);
  const uint64_t* __restrict__ keys = ctl->in_sort.result;
  int32_t* __restrict__ in_nbr = ctl->in_nbr;
  int32_t* __restrict__ ustart = ctl->udst_start;
  if (base == 0 && threadIdx.x == 0) ustart[Vd] = (int32_t)E;
  // a dst-run index is always below Vd; anything else is recorded, not written
  for (uint32_t k = base + threadIdx.x; k < end; k += blockDim.x) {
    const uint64_t key = __ldcs(keys + k);
    const uint32_t d = (uint32_t)(key >> 32);
    if (k == 0 || d != (uint32_t)(keys[k - 1] >> 32)) {
      if (d < Vd) ustart[d] = (int32_t)k;
      else atomicOr(&ctl->err, kErrRemap);
    }
    in_nbr[k] = (int32_t)(uint32_t)key;
  }
}

void launch_dst_runs(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (L.row_slots) k_dst_runs<<<L.row_slots, 256, 0, s>>>(L.ctls, L.rows, counter);
}

// ----------------------------------------------------------- node merge ---
// node_ids = usrc U udst (both ascending).  Merge path over the two lists,
// with a src item placed before an equal dst item; a dst item equal to the
// src item before it is the same node and is dropped.  For every node the
// merge cursor (i, j) (src items and dst items consumed before it) gives
//   out_off[r] = usrc_start[i]   and   in_off[r] = udst_start[j],
// which holds for nodes in both lists and for nodes in only one of them.
// Also src_rank[i] and dst_rank[j]: the node index of each list entry.
__device__ __forceinline__ uint32_t merge_path(const int32_t* __restrict__ a, uint32_t na,
                                               const int32_t* __restrict__ b, uint32_t nb,
                                               uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0;
  uint32_t hi = diag < na ? diag : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void merge_tile(Ctl* __restrict__ ctl, uint32_t tile, uint32_t* s_sw,
                                           uint64_t* s_prefix) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t Vs = ctl->Vs, Vd = ctl->Vd, M = Vs + Vd;
  const uint32_t ntiles = (M + kMergeTile - 1) / kMergeTile;
  if (tile >= ntiles) return;
  const int32_t* __restrict__ usrc = ctl->usrc;
  const int32_t* __restrict__ udst = ctl->udst;
  const uint32_t k0 = tile * (uint32_t)kMergeTile + tid * kMergeItems;
  int32_t x[kMergeItems];
  uint32_t ci[kMergeItems], cj[kMergeItems];
  uint32_t emit = 0, from_src = 0, cnt = 0, used = 0;
  if (k0 < M) {
    uint32_t i = merge_path(usrc, Vs, udst, Vd, k0);
    uint32_t j = k0 - i;
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) {
      if (k0 + q >= M) break;
      used |= 1u << q;
      const bool take_s = i < Vs && (j >= Vd || usrc[i] <= udst[j]);
      ci[q] = i;
      cj[q] = j;
      if (take_s) {
        x[q] = usrc[i];
        emit |= 1u << q;
        from_src |= 1u << q;
        ++i;
      } else {
        x[q] = udst[j];
        if (i == 0 || usrc[i - 1] != x[q]) emit |= 1u << q;
        ++j;
      }
    }
    cnt = __popc(emit);
  }
  uint32_t total;
  const uint32_t local = block_exclusive_sum<kScanThreads>(cnt, s_sw, total);
  if (warp == 0) {
    const uint64_t excl = scan_prefix(ctl->scan_status[2], chunks_of(ctl, 2), tile, ntiles,
                                      pack2(0, total), &ctl->err);
    if (lane == 0) {
      *s_prefix = excl;
      if (tile == ntiles - 1) {
        const uint32_t V = unpackB(excl) + total;
        ctl->V = V;
        ctl->out_off[V] = (int64_t)ctl->E;
        ctl->in_off[V] = (int64_t)ctl->E;
      }
    }
  }
  __syncthreads();
  uint32_t r = unpackB(*s_prefix) + local;  // nodes emitted before this item
  const int32_t* __restrict__ us = ctl->usrc_start;
  const int32_t* __restrict__ ud = ctl->udst_start;
#pragma unroll
  for (int q = 0; q < kMergeItems; ++q) {
    if (!((used >> q) & 1u)) continue;
    const bool e = (emit >> q) & 1u;
    if ((from_src >> q) & 1u) {
      ctl->src_rank[ci[q]] = (int32_t)r;
    } else {
      // a dropped dst item is the node emitted just before it
      ctl->dst_rank[cj[q]] = (int32_t)(e ? r : r - 1);
    }
    if (e) {
      ctl->node_ids[r] = x[q];
      ctl->out_off[r] = us[ci[q]];
      ctl->in_off[r] = ud[cj[q]];
      ++r;
    }
  }
}

// Persistent: blocks claim merge slots in order until none is left.
__global__ void __launch_bounds__(kScanThreads)
    k_merge(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ uint32_t s_sw[kWarps + 1];
  __shared__ uint64_t s_prefix;
  __shared__ Claim s_cl;
  while (true) {
    if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
    __syncthreads();
    if (!s_cl.valid) return;
    merge_tile(ctls + s_cl.seg, s_cl.tile, s_sw, &s_prefix);
    __syncthreads();
  }
}

// Slot maps of phase 2 from the sizes phase 1 left in each control block:
// merge tiles cover Vs + Vd items, block-table pieces cover max(Vs, Vd) / 32
// words.  One block; segments in order.
__global__ void k_phase2_maps(Ctl* __restrict__ ctls, uint32_t nseg, uint32_t* merge_start,
                              uint32_t* block_start) {
  __shared__ uint32_t s_sw[32 + 1], s_sw2[32 + 1];
  __shared__ uint32_t carry_m, carry_b;
  if (threadIdx.x == 0) {
    carry_m = 0;
    carry_b = 0;
  }
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nseg; b0 += blockDim.x) {
    const uint32_t sidx = b0 + threadIdx.x;
    uint32_t mt = 0, bt = 0;
    if (sidx < nseg) {
      const Ctl* c = ctls + sidx;
      mt = (c->Vs + c->Vd + kMergeTile - 1) / kMergeTile;
      const uint32_t words = ((c->Vs > c->Vd ? c->Vs : c->Vd) + 31) >> kBlkShift;
      bt = (words + kScanTile - 1) / kScanTile;
    }
    uint32_t tm, tb;
    const uint32_t em = block_exclusive_sum<1024>(mt, s_sw, tm);
    const uint32_t eb = block_exclusive_sum<1024>(bt, s_sw2, tb);
    if (sidx < nseg) {
      merge_start[sidx] = carry_m + em;
      block_start[sidx] = carry_b + eb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_m += tm;
      carry_b += tb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    merge_start[nseg] = carry_m;
    block_start[nseg] = carry_b;
  }
}

void launch_phase2_maps(const Launch& L, cudaStream_t s) {
  k_phase2_maps<<<1, 1024, 0, s>>>(L.ctls, L.nseg, const_cast<uint32_t*>(L.merge.start),
                                   const_cast<uint32_t*>(L.blocks.start));
}

static uint32_t persistent_grid(uint32_t per_sm) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (uint32_t)sms * per_sm;
}

void launch_merge(const Launch& L, uint32_t* counter, cudaStream_t s) {
  k_merge<<<persistent_grid(8), kScanThreads, 0, s>>>(L.ctls, L.merge, counter);
}

// ---------------------------------------------------------- block tables --
// blk[k] = map[32k], with kBlkDense set when the 32 entries from 32k are
// consecutive node indices (no node of the other kind lies between them);
// then map[j] = (blk[j >> 5] & ~kBlkDense) + (j & 31) without reading map.
__global__ void __launch_bounds__(256)
    k_rank_blocks(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  while (true) {
  if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t Vs = ctl->Vs, Vd = ctl->Vd;
  const uint32_t ns = (Vs + 31) >> kBlkShift, nd = (Vd + 31) >> kBlkShift;
  const uint32_t k0 = s_cl.tile * (uint32_t)kScanTile;
  const uint32_t k1 = k0 + (uint32_t)kScanTile;
  for (uint32_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    if (k < ns) {
      const uint32_t a = k << kBlkShift, e = min(a + 32, Vs) - 1;
      const int32_t r0 = ctl->src_rank[a], r1 = ctl->src_rank[e];
      ctl->src_blk[k] = (uint32_t)r0 | ((uint32_t)(r1 - r0) == e - a ? kBlkDense : 0u);
    }
    if (k < nd) {
      const uint32_t a = k << kBlkShift, e = min(a + 32, Vd) - 1;
      const int32_t r0 = ctl->dst_rank[a], r1 = ctl->dst_rank[e];
      ctl->dst_blk[k] = (uint32_t)r0 | ((uint32_t)(r1 - r0) == e - a ? kBlkDense : 0u);
    }
  }
  __syncthreads();
  }
}

void launch_rank_blocks(const Launch& L, uint32_t* counter, cudaStream_t s) {
  k_rank_blocks<<<persistent_grid(4), 256, 0, s>>>(L.ctls, L.blocks, counter);
}

// ---------------------------------------------------------------- remap ---
// out_nbr: dst-run index -> node index; in_nbr: source-run index -> node
// index.  Eight edges per thread; the block tables are small enough to stay
// in L2, and the full maps are read only inside blocks with a gap.
__device__ __forceinline__ int32_t map_index(const uint32_t* __restrict__ blk,
                                             const int32_t* __restrict__ map, uint32_t len,
                                             uint32_t j, uint32_t* err) {
  if (j >= len) {  // never for a correct run index: recorded, not read
    atomicOr(err, kErrRemap);
    return 0;
  }
  const uint32_t p = __ldg(blk + (j >> kBlkShift));
  if (p & kBlkDense) return (int32_t)((p & ~kBlkDense) + (j & 31));
  return __ldg(map + j);
}

// One direction of the remap over entries [base, end), in place.
__device__ __forceinline__ void remap_range(int32_t* __restrict__ a, uint32_t base, uint32_t end,
                                            const uint32_t* __restrict__ blk,
                                            const int32_t* __restrict__ map, uint32_t len,
                                            uint32_t* err) {
  for (uint32_t e = base + threadIdx.x * 4; e < end; e += blockDim.x * 4) {
    if (e + 4 <= end && (e & 3) == 0) {
      int4 x = __ldcs(reinterpret_cast<const int4*>(a + e));
      x.x = map_index(blk, map, len, (uint32_t)x.x, err);
      x.y = map_index(blk, map, len, (uint32_t)x.y, err);
      x.z = map_index(blk, map, len, (uint32_t)x.z, err);
      x.w = map_index(blk, map, len, (uint32_t)x.w, err);
      __stcs(reinterpret_cast<int4*>(a + e), x);
    } else {
      for (uint32_t q = e; q < min(e + 4, end); ++q)
        a[q] = map_index(blk, map, len, (uint32_t)a[q], err);
    }
  }
}

// When every node is a source (Vs == V) the source-run index already is the
// node index and in_nbr is left as it is; likewise out_nbr when Vd == V.
__global__ void __launch_bounds__(256)
    k_remap(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t E = ctl->E, V = ctl->V, Vs = ctl->Vs, Vd = ctl->Vd;
  const uint32_t base = s_cl.tile * (uint32_t)kScanTile;
  if (base >= E) return;
  const uint32_t end = min(E, base + (uint32_t)kScanTile);
  uint32_t* err = &ctl->err;
  if (Vd != V) remap_range(ctl->out_nbr, base, end, ctl->dst_blk, ctl->dst_rank, Vd, err);
  if (Vs != V) remap_range(ctl->in_nbr, base, end, ctl->src_blk, ctl->src_rank, Vs, err);
}

void launch_remap(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (L.row_slots) k_remap<<<L.row_slots, 256, 0, s>>>(L.ctls, L.rows, counter);
}

// -------------------------------------------------------------- degrees ---
__global__ void k_degrees(const int32_t* __restrict__ node_ids, const int64_t* __restrict__ off,
                          uint32_t V, const int32_t* __restrict__ q, uint32_t n,
                          int64_t* __restrict__ deg) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int32_t x = q[t];
    uint32_t lo = 0, hi = V;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (node_ids[mid] < x) lo = mid + 1;
      else hi = mid;
    }
    deg[t] = (lo < V && node_ids[lo] == x) ? off[lo + 1] - off[lo] : -1;
  }
}

void launch_degrees(const int32_t* node_ids, const int64_t* off, uint32_t V, const int32_t* ids,
                    uint32_t n, int64_t* deg, cudaStream_t s) {
  if (n == 0) return;
  uint32_t grid = (n + 255) / 256;
  if (grid > 8192) grid = 8192;
  k_degrees<<<grid, 256, 0, s>>>(node_ids, off, V, ids, n, deg);
}

// ---------------------------------------------------------------- top-k ---
// Nodes of largest degree, ties broken by smaller ID.  Each node gets the key
// (degree << 32) | (0xFFFFFFFF - index): larger is better, and node index
// order is ID order.  The k-th largest key is found by an MSD radix select
// (8 digit rounds), the k keys at or above it are gathered, and one block
// sorts them.
struct TopkState {
  uint64_t prefix;      // digits of the k-th key fixed so far
  uint32_t remaining;   // rank of the k-th key among keys matching prefix
  uint32_t count;       // gathered keys
  uint32_t hist[kRadix];
};

__device__ __forceinline__ uint64_t topk_key(const int64_t* off, uint32_t r) {
  const uint64_t d = (uint64_t)(off[r + 1] - off[r]);
  return (d << 32) | (0xFFFFFFFFu - r);
}

__global__ void k_topk_hist(const int64_t* __restrict__ off, uint32_t V, TopkState* st,
                            int round) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int sh = 56 - 8 * round;
  const uint64_t pre = st->prefix;
  const uint64_t hi_mask = round == 0 ? 0ull : (~0ull << (64 - 8 * round));
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < V; r += gridDim.x * blockDim.x) {
    const uint64_t k = topk_key(off, r);
    if ((k & hi_mask) == pre) atomicAdd(&h[(k >> sh) & 0xFF], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_topk_pick(TopkState* st, int round) {
  // one thread: walk digits from the top to find the bucket of the k-th key
  if (threadIdx.x != 0) return;
  const int sh = 56 - 8 * round;
  uint32_t rem = st->remaining;
  for (int d = kRadix - 1; d >= 0; --d) {
    const uint32_t c = st->hist[d];
    if (rem <= c) {
      st->prefix |= (uint64_t)d << sh;
      break;
    }
    rem -= c;
  }
  st->remaining = rem;
  for (int d = 0; d < kRadix; ++d) st->hist[d] = 0;
}

__global__ void k_topk_gather(const int64_t* __restrict__ off, uint32_t V, TopkState* st,
                              uint64_t* out, uint32_t k) {
  const uint64_t thr = st->prefix;  // the k-th largest key; keys are distinct
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < V; r += gridDim.x * blockDim.x) {
    const uint64_t key = topk_key(off, r);
    if (key >= thr) {
      const uint32_t slot = atomicAdd(&st->count, 1u);
      if (slot < k) out[slot] = key;
    }
  }
}

constexpr int kTopkMax = 4096;
__global__ void __launch_bounds__(1024) k_topk_sort(const int32_t* __restrict__ node_ids,
                                                    const uint64_t* in, uint32_t k,
                                                    int32_t* ids, int64_t* degs) {
  __shared__ uint64_t s[kTopkMax];
  uint32_t p2 = 1;
  while (p2 < k) p2 <<= 1;
  for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) s[i] = i < k ? in[i] : 0;
  __syncthreads();
  // bitonic sort, descending
  for (uint32_t size = 2; size <= p2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) {
        const uint32_t j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const uint64_t a = s[i], b = s[j];
          if (desc ? (a < b) : (a > b)) {
            s[i] = b;
            s[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    const uint64_t key = s[i];
    const uint32_t r = 0xFFFFFFFFu - (uint32_t)key;
    ids[i] = node_ids[r];
    degs[i] = (int64_t)(key >> 32);
  }
}

size_t topk_scratch_bytes(uint32_t V, uint32_t k) {
  (void)V;
  return sizeof(TopkState) + 16 + sizeof(uint64_t) * (size_t)(k ? k : 1);
}

int launch_topk(const int32_t* node_ids, const int64_t* off, uint32_t V, uint32_t k,
                int32_t* d_ids, int64_t* d_degs, void* d_scratch, size_t scratch_bytes,
                cudaStream_t s) {
  if (k == 0 || V == 0) return 0;
  if (k > (uint32_t)kTopkMax || k > V) return -1;
  if (scratch_bytes < topk_scratch_bytes(V, k)) return -1;
  TopkState* st = reinterpret_cast<TopkState*>(d_scratch);
  uint64_t* keys = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(st + 1) + 15) & ~(uintptr_t)15);
  TopkState init{};
  init.prefix = 0;
  init.remaining = k;
  init.count = 0;
  cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  uint32_t grid = (V + 255) / 256;
  if (grid > 2048) grid = 2048;
  for (int round = 0; round < 8; ++round) {
    k_topk_hist<<<grid, kRadix, 0, s>>>(off, V, st, round);
    k_topk_pick<<<1, 32, 0, s>>>(st, round);
  }
  k_topk_gather<<<grid, 256, 0, s>>>(off, V, st, keys, k);
  k_topk_sort<<<1, 1024, 0, s>>>(node_ids, keys, k, d_ids, d_degs);
  return 0;
}

}  // namespace ringo
