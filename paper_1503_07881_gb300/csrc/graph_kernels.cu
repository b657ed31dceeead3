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
  // a chunk of these scans covers at most 32 tiles of 4096 items
  static_assert(kChunkTiles * kScanTile <= (1 << 17), "chunk sums fit 24 bits");
  return ScanChunks{ctl->scan_chunk_agg[i], ctl->scan_chunk_inc[i], ctl->scan_chunk_cnt[i],
                    ctl->spin_limit, 1u};
}
}  // namespace

// ------------------------------------------------------------------ K3 ----
// Input: the out-sorted keys (bias(src) << 32 | dst-run index), n_rows of
// them.  A key that differs from its predecessor is a distinct edge e; a key
// whose src differs is the start of a source run s.  Outputs:
//   in-sort keys  spare[e]   = dst-run index << 32 | s_index(src)
//   out_nbr[e]               = dst-run index (turned into a node index later)
//   usrc[s], usrc_start[s]   = src ID and its first edge; usrc_start[Vs] = E
//   in_sort.hist             = digit histograms of the in-sort passes, RB-bit
//                              digits of the dst-run index (pass p, digit d
//                              at [(p << RB) + d])
template <int RB>
__global__ void __launch_bounds__(kScanThreads, 6)
    k_dedup(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  constexpr int R = 1 << RB;
  __shared__ uint64_t s_keys[kScanTile];  // the tile, read once, coalesced
  __shared__ uint32_t s_hist[kInPasses][R];
  __shared__ uint32_t s_we[kWarps], s_ws[kWarps];
  __shared__ uint64_t s_prefix, s_before;
  __shared__ Claim s_cl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) claim_slot(m, counter, &s_cl);
  for (int i = tid; i < kInPasses * R; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t tile = s_cl.tile;
  const uint32_t n = ctl->n_rows;
  const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (tile >= ntiles) return;
  const uint64_t* __restrict__ keys = ctl->out_sort.result;
  const uint32_t base = tile * (uint32_t)kScanTile;
  const uint32_t cnt = min((uint32_t)kScanTile, n - base);
  // in-sort digit positions that can vary: dst-run indices are below Vd
  const uint32_t Vd = ctl->Vd;
  int npos = 1;
  while (npos < kInPasses && ((Vd - 1) >> (RB * npos)) != 0) ++npos;
  for (uint32_t j = tid; j < cnt; j += kScanThreads) s_keys[j] = __ldcs(keys + base + j);
  if (tid == 0) s_before = base > 0 ? keys[base - 1] : 0;
  __syncthreads();

  const uint32_t wl = warp * (kScanItems * 32);  // the warp's first item in the tile
  const uint32_t lt = lanemask_lt();
  uint32_t he = 0, hs = 0, ce = 0, cs = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t j = wl + i * 32 + lane;
    bool h_e = false, h_s = false;
    if (j < cnt) {
      const uint64_t k = s_keys[j];
      const uint64_t p = j ? s_keys[j - 1] : s_before;
      const bool first = base + j == 0;
      h_e = first || k != p;
      h_s = first || (k >> 32) != (p >> 32);
    }
    ce += __popc(__ballot_sync(0xFFFFFFFFu, h_e));
    cs += __popc(__ballot_sync(0xFFFFFFFFu, h_s));
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
        // positions that cannot vary hold every edge in digit 0
        for (int p = npos; p < kInPasses; ++p) ctl->in_sort.hist[p << RB] = E;
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
  const int top = npos - 1;
  uint32_t ce2 = 0, cs2 = 0;  // heads of earlier items of this warp (positions recomputed)
#pragma unroll 4
  for (int i = 0; i < kScanItems; ++i) {
    const bool h = (he >> i) & 1u;
    const bool head_s = (hs >> i) & 1u;
    const uint32_t emask = __ballot_sync(0xFFFFFFFFu, h);
    const uint32_t smask = __ballot_sync(0xFFFFFFFFu, head_s);
    const uint32_t e = e0 + ce2 + __popc(emask & lt);
    const uint32_t s = s0 + cs2 + __popc(smask & lt);
    ce2 += __popc(emask);
    cs2 += __popc(smask);
    if (!h) continue;
    const uint64_t k = s_keys[wl + i * 32 + lane];
    const uint32_t db = (uint32_t)k;
    // the highest varying position takes few values: one add per value per
    // warp instead of up to 32 colliding adds on one counter
    const uint32_t td = (db >> (RB * top)) & (R - 1u);
    const uint32_t peers = __match_any_sync(emask, td);
    if (lane == 31 - __clz(peers)) atomicAdd(&s_hist[top][td], (uint32_t)__popc(peers));
    const uint32_t sidx = head_s ? s : s - 1;
    ekeys[e] = ((uint64_t)db << 32) | sidx;
    out_nbr[e] = (int32_t)db;
#pragma unroll
    for (int p = 0; p < kInPasses - 1; ++p)  // fixed trip count: predicated, no loop branch
      if (p < top) atomicAdd(&s_hist[p][(db >> (RB * p)) & (R - 1u)], 1u);
    if (head_s) {
      usrc[s] = unbias((uint32_t)(k >> 32));
      usrc_start[s] = (int32_t)e;
    }
  }
  __syncthreads();
  for (int i = tid; i < kInPasses * R; i += kScanThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(&ctl->in_sort.hist[0] + i, c);
  }
}

void launch_dedup(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (!L.row_slots) return;
  if (L.opts.in_digit_bits == 9)
    k_dedup<9><<<L.row_slots, kScanThreads, 0, s>>>(L.ctls, L.rows, counter);
  else
    k_dedup<8><<<L.row_slots, kScanThreads, 0, s>>>(L.ctls, L.rows, counter);
}

// ------------------------------------------------------------- dst rank ---
// Runs between out-sort passes 3 and 4, when the keys are in dst order.
// Each key's dst is replaced by its destination-run index (the rank of the
// dst among the distinct dst values), which keeps the key order; the run
// heads give udst[], the distinct destination IDs in ascending order.
// Reads rank_step.in (or packs from the columns when every dst pass was
// trivial) and writes rank_step.out.  Single-pass compaction count with
// decoupled look-back.
__global__ void __launch_bounds__(kScanThreads, 6)
    k_dst_rank(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter, uint32_t ahead_slots) {
  __shared__ uint64_t s_keys[kScanTile];  // the tile, read once, coalesced
  __shared__ uint64_t s_before;           // the key just before the tile
  __shared__ uint32_t s_w[kWarps];
  __shared__ uint64_t s_prefix;
  __shared__ Claim s_cl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    claim_slot(m, counter, &s_cl);
    // a single table: the tile one wave of resident blocks ahead goes to L2
    // already, so that block's loads do not wait on DRAM
    const uint32_t ahead = s_cl.slot + ahead_slots;
    if (m.nseg == 1 && ahead < __ldg(m.start + 1)) {
      const uint32_t n0 = ctls->n_rows, b0 = ahead * (uint32_t)kScanTile;
      const uint64_t* in0 = ctls->rank_step.in;
      if (in0 && b0 < n0) {
        const uint32_t k = min((uint32_t)kScanTile, n0 - b0) & ~1u;
        if (k) bulk_prefetch_l2(in0 + b0, k * 8u);
      }
    }
  }
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
  const uint32_t base = tile * (uint32_t)kScanTile;
  const uint32_t cnt = min((uint32_t)kScanTile, n - base);
  if (in) {
    for (uint32_t j = tid; j < cnt; j += kScanThreads) s_keys[j] = __ldcs(in + base + j);
  } else {
    for (uint32_t j = tid; j < cnt; j += kScanThreads) s_keys[j] = key_at(base + j);
  }
  if (tid == 0) s_before = base > 0 ? key_at(base - 1) : 0;
  __syncthreads();
  const uint32_t wl = warp * (kScanItems * 32);  // the warp's first item in the tile
  const uint32_t lt = lanemask_lt();
  uint32_t hd = 0, cd = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t j = wl + i * 32 + lane;
    bool h = false;
    if (j < cnt) {
      const uint64_t k = s_keys[j];
      const uint64_t p = j ? s_keys[j - 1] : s_before;
      h = (base + j == 0) || (uint32_t)k != (uint32_t)p;
    }
    cd += __popc(__ballot_sync(0xFFFFFFFFu, h));
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
  uint32_t cd2 = 0;  // heads of earlier items of this warp
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const bool h = (hd >> i) & 1u;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, h);
    const uint32_t dl = cd2 + __popc(b & lt);
    cd2 += __popc(b);
    const uint32_t j = wl + i * 32 + lane;
    if (j >= cnt) continue;
    const uint64_t k = s_keys[j];
    const uint32_t r = d0 + dl + (h ? 0u : 0xFFFFFFFFu);  // inclusive count - 1
    __stcs(out + base + j, (k & 0xFFFFFFFF00000000ull) | r);
    if (h) udst[r] = unbias((uint32_t)k);
  }
}

void launch_dst_rank(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (!L.row_slots) return;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t ahead = 6u * (uint32_t)sms;  // six blocks resident per SM
  k_dst_rank<<<L.row_slots, kScanThreads, 0, s>>>(L.ctls, L.rows, counter, ahead);
}

// ------------------------------------------------------------------ K5 ----
// Input: the in-sorted keys (dst-run index << 32 | source-run index), E of
// them, in (dst, src) order.  Writes in_nbr[k] = the node index of the
// source run (phase 2 has built the source-run -> node map) and, at each
// change of dst-run index d, the run's first in-edge udst_start[d] = k
// (udst_start[Vd] = E, in_off[V] = E).  Every dst-run index occurs, so no
// compaction is needed.
__device__ __forceinline__ int32_t map_index(const uint32_t* __restrict__ blk,
                                             const int32_t* __restrict__ map, uint32_t len,
                                             uint32_t j, uint32_t* err);

__global__ void __launch_bounds__(256)
    k_dst_runs(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t E = ctl->E, Vd = ctl->Vd, Vs = ctl->Vs, V = ctl->V;
  const uint32_t base = s_cl.tile * (uint32_t)kScanTile;
  if (base >= E) return;
  const uint32_t end = min(E, base + (uint32_t)kScanTile);
  const uint64_t* __restrict__ keys = ctl->in_sort.result;
  int32_t* __restrict__ in_nbr = ctl->in_nbr;
  int32_t* __restrict__ ustart = ctl->udst_start;
  if (base == 0 && threadIdx.x == 0) {
    ustart[Vd] = (int32_t)E;
    ctl->in_off[V] = (int64_t)E;
  }
  // when every node is a source the source-run index is the node index
  const bool ident = Vs == V;
  const uint32_t* __restrict__ blk = ctl->src_blk;
  const int32_t* __restrict__ map = ctl->src_rank;
  // a dst-run index is always below Vd; anything else is recorded, not written
  for (uint32_t k = base + threadIdx.x; k < end; k += blockDim.x) {
    const uint64_t key = __ldcs(keys + k);
    const uint32_t d = (uint32_t)(key >> 32);
    if (k == 0 || d != (uint32_t)(keys[k - 1] >> 32)) {
      if (d < Vd) ustart[d] = (int32_t)k;
      else atomicOr(&ctl->err, kErrRemap);
    }
    const uint32_t sidx = (uint32_t)key;
    __stcs(in_nbr + k, ident ? (int32_t)sidx : map_index(blk, map, Vs, sidx, &ctl->err));
  }
}

void launch_dst_runs(const Launch& L, uint32_t* counter, cudaStream_t s) {
  if (L.row_slots) k_dst_runs<<<L.row_slots, 256, 0, s>>>(L.ctls, L.rows, counter);
}

// in_off from the destination runs, after the in-sort: run j (first in-edge
// udst_start[j], node dst_rank[j]) gives in_off = udst_start[j] to its node
// and to every node between the previous run's node and it (nodes that are
// not destinations have empty in-lists); after the last run in_off = E up to
// node V.  Persistent over the merge tiles of every segment, kMergeTile runs
// a tile (a segment's tiles cover Vs + Vd >= Vd items).  A node range of
// kFillInline nodes or more is recorded (first node, last node, value) in
// usrc_start, which phase 3 does not use, and filled by k_fill_ranges, so
// that no thread writes a long range alone.
constexpr uint32_t kFillInline = 32;

__device__ __forceinline__ void fill_nodes(Ctl* __restrict__ ctl, int64_t* __restrict__ in_off,
                                           uint32_t a, uint32_t b, uint32_t v) {
  if (b - a < kFillInline) {
    for (uint32_t r = a; r <= b; ++r) in_off[r] = (int64_t)v;
    return;
  }
  // three words a range; a range holds at least kFillInline of the at most
  // 2 * n_rows nodes, so n_rows + 1 words always suffice
  const uint32_t i = atomicAdd(&ctl->n_fill, 1u);
  uint32_t* rec = reinterpret_cast<uint32_t*>(ctl->usrc_start);
  if (3ull * i + 2 < (uint64_t)ctl->n_rows + 1) {
    rec[3 * i] = a;
    rec[3 * i + 1] = b;
    rec[3 * i + 2] = v;
  } else {
    atomicOr(&ctl->err, kErrRemap);
  }
}

__global__ void __launch_bounds__(256)
    k_fill_in_off(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  while (true) {
    if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
    __syncthreads();
    if (!s_cl.valid) return;
    Ctl* __restrict__ ctl = ctls + s_cl.seg;
    const uint32_t V = ctl->V, Vd = ctl->Vd, E = ctl->E;
    const uint32_t j0 = s_cl.tile * (uint32_t)kMergeTile;
    const uint32_t j1 = min(Vd, j0 + (uint32_t)kMergeTile);
    int64_t* __restrict__ in_off = ctl->in_off;
    const int32_t* __restrict__ ustart = ctl->udst_start;
    const int32_t* __restrict__ drank = ctl->dst_rank;
    for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
      const uint32_t r1 = (uint32_t)drank[j];
      const uint32_t r0 = j ? (uint32_t)drank[j - 1] + 1 : 0u;
      if (r1 >= V || r0 > r1) {  // the run nodes ascend below V (never expected otherwise)
        atomicOr(&ctl->err, kErrRemap);
        continue;
      }
      fill_nodes(ctl, in_off, r0, r1, (uint32_t)ustart[j]);
      if (j == Vd - 1 && r1 + 1 < V) fill_nodes(ctl, in_off, r1 + 1, V - 1, E);
    }
    __syncthreads();
  }
}

// The node ranges k_fill_in_off recorded (long runs of nodes that are not
// destinations; rare), one warp per range.  One block per segment.
__global__ void __launch_bounds__(256) k_fill_ranges(Ctl* __restrict__ ctls) {
  Ctl* __restrict__ ctl = ctls + blockIdx.x;
  const uint32_t cap = (uint32_t)(((uint64_t)ctl->n_rows + 1) / 3);
  const uint32_t n = min(ctl->n_fill, cap);
  const uint32_t* __restrict__ rec = reinterpret_cast<const uint32_t*>(ctl->usrc_start);
  int64_t* __restrict__ in_off = ctl->in_off;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  for (uint32_t i = warp; i < n; i += warps) {
    const uint32_t a = rec[3 * i], b = rec[3 * i + 1];
    const int64_t v = (int64_t)rec[3 * i + 2];
    for (uint64_t r = (uint64_t)a + lane; r <= b; r += 32) in_off[r] = v;
  }
}

// ----------------------------------------------------------- node merge ---
// node_ids = usrc U udst (both ascending).  Merge path over the two lists,
// with a src item placed before an equal dst item; a dst item equal to the
// src item before it is the same node and is dropped.  For every node the
// merge cursor i (src items consumed before it) gives out_off[r] =
// usrc_start[i], which holds for nodes in both lists and for nodes in only
// one of them.  in_off is written after the in-sort, by k_dst_runs.
// Also src_rank[i] and dst_rank[j]: the node index of each list entry.
__device__ __forceinline__ uint32_t merge_path(const int32_t* a, uint32_t na, const int32_t* b,
                                               uint32_t nb, uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0;
  uint32_t hi = diag < na ? diag : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One merge tile: kMergeTile consecutive items of the merged order, between
// the splits found by k_merge_split.
// The tile's slices of usrc / udst and of their run starts are loaded into
// shared memory (coalesced), each thread merges kMergeItems items from there,
// and the outputs are staged so that node_ids, both offset arrays and both
// rank maps are written coalesced.
struct MergeSmem {
  int32_t val[kMergeTile];        // usrc[i0, i1) then udst[j0, j1)
  int32_t start[kMergeTile + 1];  // usrc_start[i0, i1]
  int32_t rank[kMergeTile];       // tile-local node index of each input item
  uint32_t node[kMergeTile];      // emitted nodes: i | j << 12 | from_src << 24 (local)
  uint32_t sw[kWarps + 1];
  int32_t prev;                   // usrc[i0 - 1]
  uint32_t has_prev;
  uint64_t prefix;
};

// The merge path splits of every merge tile of every table, before the
// merge: one binary search per tile start, all of them in parallel.  The
// splits go to the in-CSR neighbour array, which only phase 3 writes.
__global__ void __launch_bounds__(256)
    k_merge_split(Ctl* __restrict__ ctls, SegMap m) {
  const uint32_t total = __ldg(m.start + m.nseg);
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += gridDim.x * blockDim.x) {
    const uint32_t sidx = seg_of(m, g);
    Ctl* __restrict__ ctl = ctls + sidx;
    const uint32_t t = g - __ldg(m.start + sidx);
    const uint32_t Vs = ctl->Vs, Vd = ctl->Vd;
    const uint32_t diag = t * (uint32_t)kMergeTile;
    if (diag >= Vs + Vd) continue;
    merge_splits(ctl)[t] = merge_path(ctl->usrc, Vs, ctl->udst, Vd, diag);
  }
}

__device__ __forceinline__ void merge_tile(Ctl* __restrict__ ctl, uint32_t tile, MergeSmem& S) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t Vs = ctl->Vs, Vd = ctl->Vd, M = Vs + Vd;
  const uint32_t ntiles = (M + kMergeTile - 1) / kMergeTile;
  if (tile >= ntiles) return;
  const int32_t* __restrict__ usrc = ctl->usrc;
  const int32_t* __restrict__ udst = ctl->udst;
  const uint32_t k0 = tile * (uint32_t)kMergeTile;
  const uint32_t k1 = min(k0 + (uint32_t)kMergeTile, M);
  const uint32_t* __restrict__ split = merge_splits(ctl);
  const uint32_t i0 = split[tile];
  const uint32_t i1 = tile + 1 < ntiles ? split[tile + 1] : Vs;
  const uint32_t j0 = k0 - i0, j1 = k1 - i1;
  const uint32_t na = i1 - i0, nb = j1 - j0;
  const int32_t* __restrict__ us = ctl->usrc_start;
  for (uint32_t t = tid; t < na; t += kScanThreads) S.val[t] = usrc[i0 + t];
  for (uint32_t t = tid; t < nb; t += kScanThreads) S.val[na + t] = udst[j0 + t];
  for (uint32_t t = tid; t <= na; t += kScanThreads) S.start[t] = us[i0 + t];
  if (tid == 0) {
    S.has_prev = i0 > 0 ? 1u : 0u;
    S.prev = i0 > 0 ? usrc[i0 - 1] : 0;
  }
  __syncthreads();
  const int32_t* sa = S.val;
  const int32_t* sb = S.val + na;
  const uint32_t nloc = na + nb;
  const uint32_t d0 = tid * kMergeItems;
  uint32_t lij[kMergeItems];  // local cursors i | j << 16 (each at most 2048)
  uint32_t emit = 0, from_src = 0, used = 0;
  if (d0 < nloc) {
    uint32_t i = merge_path(sa, na, sb, nb, d0);
    uint32_t j = d0 - i;
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) {
      if (d0 + q >= nloc) break;
      used |= 1u << q;
      lij[q] = i | (j << 16);
      if (i < na && (j >= nb || sa[i] <= sb[j])) {
        emit |= 1u << q;
        from_src |= 1u << q;
        ++i;
      } else {
        // a dst item equal to the src item before it is the same node
        const bool has = i > 0 || S.has_prev;
        const int32_t before = i > 0 ? sa[i - 1] : S.prev;
        if (!(has && before == sb[j])) emit |= 1u << q;
        ++j;
      }
    }
  }
  uint32_t total;
  const uint32_t local = block_exclusive_sum<kScanThreads>((uint32_t)__popc(emit), S.sw, total);
  if (warp == 0) {
    const uint64_t excl = scan_prefix(ctl->scan_status[2], chunks_of(ctl, 2), tile, ntiles,
                                      pack2(0, total), &ctl->err);
    if (lane == 0) {
      S.prefix = excl;
      if (tile == ntiles - 1) {
        const uint32_t V = unpackB(excl) + total;
        ctl->V = V;
        ctl->out_off[V] = (int64_t)ctl->E;
      }
    }
  }
  // stage: tile-local node index of every input item, and the emitted nodes
  int32_t r = (int32_t)local;
#pragma unroll
  for (int q = 0; q < kMergeItems; ++q) {
    if (!((used >> q) & 1u)) continue;
    const bool e = (emit >> q) & 1u;
    const uint32_t li = lij[q] & 0xFFFFu, lj = lij[q] >> 16;
    if ((from_src >> q) & 1u) {
      S.rank[li] = r;
    } else {
      S.rank[na + lj] = e ? r : r - 1;  // a dropped dst item: the node just before
    }
    if (e) {
      S.node[r] = li | (lj << 12) | (((from_src >> q) & 1u) << 24);
      ++r;
    }
  }
  __syncthreads();
  const uint32_t r0 = unpackB(S.prefix);
  int32_t* __restrict__ node_ids = ctl->node_ids;
  int64_t* __restrict__ out_off = ctl->out_off;
  for (uint32_t t = tid; t < total; t += kScanThreads) {
    const uint32_t p = S.node[t];
    const uint32_t i = p & 0xFFFu, j = (p >> 12) & 0xFFFu;
    node_ids[r0 + t] = (p >> 24) ? sa[i] : sb[j];
    out_off[r0 + t] = S.start[i];
  }
  int32_t* __restrict__ src_rank = ctl->src_rank;
  int32_t* __restrict__ dst_rank = ctl->dst_rank;
  for (uint32_t t = tid; t < na; t += kScanThreads) src_rank[i0 + t] = (int32_t)r0 + S.rank[t];
  for (uint32_t t = tid; t < nb; t += kScanThreads) dst_rank[j0 + t] = (int32_t)r0 + S.rank[na + t];
}

// Persistent: blocks claim merge slots in order until none is left.
__global__ void __launch_bounds__(kScanThreads, 6)
    k_merge(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ MergeSmem S;
  __shared__ Claim s_cl;
  while (true) {
    if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
    __syncthreads();
    if (!s_cl.valid) return;
    merge_tile(ctls + s_cl.seg, s_cl.tile, S);
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

void launch_merge_split(const Launch& L, cudaStream_t s) {
  k_merge_split<<<persistent_grid(8), 256, 0, s>>>(L.ctls, L.merge);
}

void launch_merge(const Launch& L, uint32_t* counter, cudaStream_t s) {
  k_merge<<<persistent_grid(6), kScanThreads, 0, s>>>(L.ctls, L.merge, counter);
}

// ---------------------------------------------------------- block tables --
__device__ __forceinline__ void add_step(Ctl* ctl, uint32_t j, uint32_t off) {
  const uint32_t i = atomicAdd(&ctl->n_steps, 1u);
  if (i < (uint32_t)kMaxSteps) {
    ctl->step_j[i] = j;
    ctl->step_off[i] = off;
  }
}

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
      const bool dense = (uint32_t)(r1 - r0) == e - a;
      ctl->dst_blk[k] = (uint32_t)r0 | (dense ? kBlkDense : 0u);
      // steps of dst_rank[j] - j: at the block's start, and inside a block
      // that is not dense (looked at only while the list can still be used)
      const uint32_t off0 = (uint32_t)r0 - a;
      const uint32_t prev = a ? (uint32_t)ctl->dst_rank[a - 1] - (a - 1) : 0u;
      if (off0 != prev) add_step(ctl, a, off0);
      if (!dense && *(volatile uint32_t*)&ctl->n_steps <= (uint32_t)kMaxSteps) {
        uint32_t last = off0;
        for (uint32_t j = a + 1; j <= e; ++j) {
          const uint32_t off = (uint32_t)ctl->dst_rank[j] - j;
          if (off != last) add_step(ctl, j, off);
          last = off;
        }
      }
    }
  }
  __syncthreads();
  }
}

// Sorts each table's step list by position (one block per table; the list
// holds at most kMaxSteps entries, so a bitonic sort in shared memory).
__global__ void __launch_bounds__(kMaxSteps) k_sort_steps(Ctl* __restrict__ ctls) {
  __shared__ uint64_t s[kMaxSteps];
  Ctl* __restrict__ ctl = ctls + blockIdx.x;
  const uint32_t n = ctl->n_steps;
  if (n < 2 || n > (uint32_t)kMaxSteps) return;
  const uint32_t t = threadIdx.x;
  s[t] = t < n ? ((uint64_t)ctl->step_j[t] << 32 | ctl->step_off[t]) : ~0ull;
  __syncthreads();
  for (uint32_t size = 2; size <= (uint32_t)kMaxSteps; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      const uint32_t o = t ^ stride;
      if (o > t) {
        const bool up = (t & size) == 0;
        const uint64_t x = s[t], y = s[o];
        if (up ? x > y : x < y) {
          s[t] = y;
          s[o] = x;
        }
      }
      __syncthreads();
    }
  }
  if (t < n) {
    ctl->step_j[t] = (uint32_t)(s[t] >> 32);
    ctl->step_off[t] = (uint32_t)s[t];
  }
}

void launch_sort_steps(const Launch& L, cudaStream_t s) {
  if (L.nseg) k_sort_steps<<<L.nseg, kMaxSteps, 0, s>>>(L.ctls);
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

// One direction of the remap over the entries [base, end) of one tile, in
// place.  A full tile is 16 entries per thread, taken as four coalesced
// 128-bit loads; all block-table words are requested before any map word,
// so each thread keeps 16 independent lookups in flight.
__device__ __forceinline__ void remap_range(int32_t* __restrict__ a, uint32_t base, uint32_t end,
                                            const uint32_t* __restrict__ blk,
                                            const int32_t* __restrict__ map, uint32_t len,
                                            uint32_t* err) {
  constexpr int kVec = kScanTile / (4 * 256);  // 128-bit words per thread
  if (end - base == (uint32_t)kScanTile && blockDim.x == 256) {
    uint32_t v[4 * kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
      const int4 x = __ldcs(reinterpret_cast<const int4*>(a + base + k * 1024) + threadIdx.x);
      v[4 * k] = (uint32_t)x.x;
      v[4 * k + 1] = (uint32_t)x.y;
      v[4 * k + 2] = (uint32_t)x.z;
      v[4 * k + 3] = (uint32_t)x.w;
    }
    uint32_t w[4 * kVec];
#pragma unroll
    for (int q = 0; q < 4 * kVec; ++q) w[q] = v[q] < len ? __ldg(blk + (v[q] >> kBlkShift)) : 0u;
#pragma unroll
    for (int q = 0; q < 4 * kVec; ++q) {
      if (v[q] >= len) {  // never for a correct run index: recorded, not read
        atomicOr(err, kErrRemap);
        v[q] = 0;
      } else if (w[q] & kBlkDense) {
        v[q] = (w[q] & ~kBlkDense) + (v[q] & 31);
      } else {
        v[q] = (uint32_t)__ldg(map + v[q]);
      }
    }
#pragma unroll
    for (int k = 0; k < kVec; ++k)
      __stcs(reinterpret_cast<int4*>(a + base + k * 1024) + threadIdx.x,
             make_int4((int)v[4 * k], (int)v[4 * k + 1], (int)v[4 * k + 2], (int)v[4 * k + 3]));
    return;
  }
  for (uint32_t e = base + threadIdx.x; e < end; e += blockDim.x)
    a[e] = map_index(blk, map, len, (uint32_t)a[e], err);
}

// out_nbr only (k_dst_runs writes in_nbr in its final form).  When every
// node is a destination (Vd == V) the dst-run index already is the node
// index and out_nbr is left as it is.
__global__ void __launch_bounds__(256)
    k_remap(Ctl* __restrict__ ctls, SegMap m, uint32_t* counter) {
  __shared__ Claim s_cl;
  if (threadIdx.x == 0) claim_slot(m, counter, &s_cl);
  __syncthreads();
  if (!s_cl.valid) return;
  Ctl* __restrict__ ctl = ctls + s_cl.seg;
  const uint32_t E = ctl->E, V = ctl->V, Vd = ctl->Vd;
  const uint32_t base = s_cl.tile * (uint32_t)kScanTile;
  if (base >= E) return;
  const uint32_t end = min(E, base + (uint32_t)kScanTile);
  uint32_t* err = &ctl->err;
  if (Vd == V) return;
  const uint32_t ns = ctl->n_steps;
  if (ns > (uint32_t)kMaxSteps || blockDim.x != 256) {
    remap_range(ctl->out_nbr, base, end, ctl->dst_blk, ctl->dst_rank, Vd, err);
    return;
  }
  // few steps: node = j + the difference of the last step at or before j,
  // found by a binary search of the sorted list in shared memory
  __shared__ uint32_t s_j[kMaxSteps], s_off[kMaxSteps];
  for (uint32_t t = threadIdx.x; t < ns; t += blockDim.x) {
    s_j[t] = ctl->step_j[t];
    s_off[t] = ctl->step_off[t];
  }
  __syncthreads();
  int32_t* __restrict__ a = ctl->out_nbr;
  auto node_of = [&](uint32_t j) -> uint32_t {
    uint32_t lo = 0, hi = ns;  // steps [0, lo) are at or before j
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_j[mid] <= j) lo = mid + 1;
      else hi = mid;
    }
    return j + (lo ? s_off[lo - 1] : 0u);
  };
  if (end - base == (uint32_t)kScanTile) {
    constexpr int kVec = kScanTile / (4 * 256);
    int4 x[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k)
      x[k] = __ldcs(reinterpret_cast<const int4*>(a + base + k * 1024) + threadIdx.x);
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
      uint32_t v[4] = {(uint32_t)x[k].x, (uint32_t)x[k].y, (uint32_t)x[k].z, (uint32_t)x[k].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (v[q] >= Vd) {  // never for a correct run index: recorded, not mapped
          atomicOr(err, kErrRemap);
          v[q] = 0;
        } else {
          v[q] = node_of(v[q]);
        }
      }
      __stcs(reinterpret_cast<int4*>(a + base + k * 1024) + threadIdx.x,
             make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]));
    }
    return;
  }
  for (uint32_t e = base + threadIdx.x; e < end; e += blockDim.x) {
    const uint32_t j = (uint32_t)a[e];
    if (j >= Vd) {
      atomicOr(err, kErrRemap);
      a[e] = 0;
    } else {
      a[e] = (int32_t)node_of(j);
    }
  }
}

void launch_fill_in_off(const Launch& L, uint32_t* counter, cudaStream_t s) {
  k_fill_in_off<<<persistent_grid(8), 256, 0, s>>>(L.ctls, L.merge, counter);
  if (L.nseg) k_fill_ranges<<<L.nseg, 256, 0, s>>>(L.ctls);
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
