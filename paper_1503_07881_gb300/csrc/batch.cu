// Base tables, selection and batched conversion (ringo_base_*, ringo_select_*,
// ringo_convert_batch, ringo_batch_*).
//
// A base table (src, dst, ts, tag) is loaded once and kept on the device,
// clustered by (tag, ts) with two stable radix sorts (the table's rows keep
// their identity through a carried row index).  A predicate (tags, [t0, t1))
// then selects, for each of its tags, one contiguous range of clustered rows,
// found by binary search.  A batch gathers every selected sub-table into one
// input array and converts all of them with one run of the multi-segment
// pipeline: per-segment control blocks, upper-bound buffers and no host
// synchronisation between the kernels, so each wave of the batch is recorded
// as one CUDA graph and launched once.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"
#include "batch_internal.h"

using namespace ringo;

namespace {

// -------------------------------------------------------------- layout ------
// Byte offsets of one segment's buffers inside three regions: one that must
// start at zero, one of scratch, one of outputs (outputs sized for the upper
// bounds V <= 2n and E <= n, so no host sync is needed before phase 2).
struct SegLayout {
  uint64_t z_st0, z_ch0, z_sc0, z_sc1, z_sc2, z_total;
  uint64_t keysA, keysB, st1, ch1, usrc, usrc_start, udst, udst_start, ranks, s_total;
  uint64_t out_nbr, in_nbr, node_ids, out_off, in_off, o_total;
  uint32_t tiles, mtiles, chunks;
};

__host__ __device__ inline uint64_t al(uint64_t x) { return (x + 255) & ~255ull; }
__host__ __device__ inline uint64_t up4(uint64_t x) { return (x + 3) & ~3ull; }
__host__ __device__ inline uint64_t nchunks(uint64_t tiles) {
  return (tiles + kChunkTiles - 1) / kChunkTiles;
}
__host__ __device__ inline uint64_t scan_region(uint64_t tiles) {
  const uint64_t c = nchunks(tiles);
  return al(8 * tiles) + 2 * al(8 * c) + al(4 * c);
}

__host__ __device__ inline SegLayout seg_layout(uint32_t n) {
  SegLayout L;
  const uint64_t tiles = (n + (uint64_t)kSortTile - 1) / kSortTile;
  const uint64_t mtiles = (2ull * n + kMergeTile - 1) / kMergeTile + 1;
  const uint64_t ch = nchunks(tiles);
  const uint64_t chunk_bytes = al(radix_chunk_bytes(ch));
  L.tiles = (uint32_t)tiles;
  L.mtiles = (uint32_t)mtiles;
  L.chunks = (uint32_t)ch;
  uint64_t o = 0;
  L.z_st0 = o; o = al(o + radix_status_bytes(tiles));
  L.z_ch0 = o; o = al(o + chunk_bytes);
  L.z_sc0 = o; o = al(o + scan_region(tiles));
  L.z_sc1 = o; o = al(o + scan_region(tiles));
  L.z_sc2 = o; o = al(o + scan_region(mtiles));
  L.z_total = o;
  o = 0;
  L.keysA = o; o = al(o + 8 * (n + 1ull));
  L.keysB = o; o = al(o + 8 * (n + 1ull));
  L.st1 = o; o = al(o + radix_status_bytes(tiles));
  L.ch1 = o; o = al(o + chunk_bytes);
  L.usrc = o; o = al(o + 4 * (n + 1ull));
  L.usrc_start = o; o = al(o + 4 * (n + 1ull));
  L.udst = o; o = al(o + 4 * (n + 1ull));
  L.udst_start = o; o = al(o + 4 * (n + 1ull));
  L.ranks = o; o = al(o + 4 * (2 * up4(n) + 2 * up4((n + 31ull) / 32)));
  L.s_total = o;
  o = 0;
  L.out_nbr = o; o = al(o + 4ull * n);
  L.in_nbr = o; o = al(o + 4ull * n);
  L.node_ids = o; o = al(o + 8ull * n);
  L.out_off = o; o = al(o + 8 * (2ull * n + 1));
  L.in_off = o; o = al(o + 8 * (2ull * n + 1));
  L.o_total = o;
  return L;
}

struct SegDesc {
  uint32_t n;
  const int32_t* src;
  const int32_t* dst;
  char* zbase;
  char* sbase;
  char* obase;
};

__device__ void place_scan_dev(Ctl* c, int i, char* p, uint64_t tiles) {
  const uint64_t ch = nchunks(tiles);
  c->scan_status[i] = (uint64_t*)p;
  p += al(8 * tiles);
  c->scan_chunk_agg[i] = (uint64_t*)p;
  p += al(8 * ch);
  c->scan_chunk_inc[i] = (uint64_t*)p;
  p += al(8 * ch);
  c->scan_chunk_cnt[i] = (uint32_t*)p;
}

// One block per segment: clear its control block and point it at its
// buffers.
__global__ void k_init_ctls(Ctl* __restrict__ ctls, const SegDesc* __restrict__ desc) {
  Ctl* c = ctls + blockIdx.x;
  static_assert(sizeof(Ctl) % sizeof(uint4) == 0, "control blocks are cleared in 16-byte words");
  uint4* w = reinterpret_cast<uint4*>(c);
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (uint32_t i = threadIdx.x; i < sizeof(Ctl) / sizeof(uint4); i += blockDim.x) w[i] = z;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const SegDesc d = desc[blockIdx.x];
  const SegLayout L = seg_layout(d.n);
  c->n_rows = d.n;
  c->src = d.src;
  c->dst = d.dst;
  c->keysA = (uint64_t*)(d.sbase + L.keysA);
  c->keysB = (uint64_t*)(d.sbase + L.keysB);
  c->status[0] = (uint32_t*)(d.zbase + L.z_st0);
  c->status[1] = (uint32_t*)(d.sbase + L.st1);
  c->status_rows = L.tiles;
  for (int r = 0; r < 2; ++r)
    place_radix_chunks(c, r, r ? d.sbase + L.ch1 : d.zbase + L.z_ch0, L.chunks);
  c->chunk_rows = L.chunks;
  place_scan_dev(c, 0, d.zbase + L.z_sc0, L.tiles);
  place_scan_dev(c, 1, d.zbase + L.z_sc1, L.tiles);
  place_scan_dev(c, 2, d.zbase + L.z_sc2, L.mtiles);
  c->usrc = (int32_t*)(d.sbase + L.usrc);
  c->usrc_start = (int32_t*)(d.sbase + L.usrc_start);
  c->udst = (int32_t*)(d.sbase + L.udst);
  c->udst_start = (int32_t*)(d.sbase + L.udst_start);
  int32_t* ranks = (int32_t*)(d.sbase + L.ranks);
  c->src_rank = ranks;
  c->dst_rank = ranks + up4(d.n);
  c->src_blk = (uint32_t*)(c->dst_rank + up4(d.n));
  c->dst_blk = c->src_blk + up4((d.n + 31ull) / 32);
  c->out_nbr = (int32_t*)(d.obase + L.out_nbr);
  c->in_nbr = (int32_t*)(d.obase + L.in_nbr);
  c->node_ids = (int32_t*)(d.obase + L.node_ids);
  c->out_off = (int64_t*)(d.obase + L.out_off);
  c->in_off = (int64_t*)(d.obase + L.in_off);
}

__global__ void k_collect(const Ctl* __restrict__ ctls, uint32_t nseg, SegResult* out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += gridDim.x * blockDim.x) {
    const Ctl* c = ctls + i;
    SegResult r;
    r.V = c->V;
    r.E = c->E;
    r.Vs = c->Vs;
    r.Vd = c->Vd;
    r.err = c->err;
    r.out_passes = c->out_sort.active_passes;
    r.in_passes = c->in_sort.active_passes;
    r.pad = 0;
    out[i] = r;
  }
}

// ------------------------------------------------------------ base load -----
__global__ void k_minmax_i64(const int64_t* __restrict__ ts, uint32_t n, long long* mm) {
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long v = ts[i];
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long a = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
    const long long b = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(mm, lo);
    atomicMax(mm + 1, hi);
  }
}

// stage 1 columns: key high word = ts - ts_min, low word = row
__global__ void k_stage1_cols(const int64_t* __restrict__ ts, const long long* mm, uint32_t n,
                              int32_t* a, int32_t* b) {
  const long long t0 = mm[0];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a[i] = (int32_t)((uint32_t)(ts[i] - t0) ^ kBias);
    b[i] = (int32_t)i;
  }
}

// stage 2 columns, in stage-1 order: key high word = tag, low word = position
__global__ void k_stage2_cols(const Ctl* __restrict__ sort1, const int32_t* __restrict__ tag,
                              uint32_t n, int32_t* a, int32_t* b, int32_t* o1) {
  const uint64_t* keys = sort1->out_sort.result;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t row = (uint32_t)keys[p];
    o1[p] = (int32_t)row;
    a[p] = tag[row < n ? row : 0];
    b[p] = (int32_t)p;
  }
}

__global__ void k_cluster_gather(const Ctl* __restrict__ sort2, const int32_t* __restrict__ o1,
                                 uint32_t n, const int32_t* __restrict__ src,
                                 const int32_t* __restrict__ dst, const int64_t* __restrict__ ts,
                                 const int32_t* __restrict__ tag, int32_t* src_c, int32_t* dst_c,
                                 int64_t* ts_c, int32_t* tag_c) {
  const uint64_t* keys = sort2->out_sort.result;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t p = (uint32_t)keys[q];
    const uint32_t row = (uint32_t)o1[p < n ? p : 0];
    const uint32_t r = row < n ? row : 0;
    src_c[q] = src[r];
    dst_c[q] = dst[r];
    ts_c[q] = ts[r];
    tag_c[q] = tag[r];
  }
}

// ------------------------------------------------------------- select -------
// first clustered row not below (tag, t)
__device__ __forceinline__ uint32_t lower_bound_tt(const int32_t* __restrict__ tag_c,
                                                   const int64_t* __restrict__ ts_c, uint32_t n,
                                                   int32_t tag, int64_t t) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const int32_t g = tag_c[mid];
    if (g < tag || (g == tag && ts_c[mid] < t)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_select(const int32_t* __restrict__ tag_c, const int64_t* __restrict__ ts_c,
                         uint32_t n, const Pair* __restrict__ pairs, uint32_t npairs,
                         uint32_t* lo, uint32_t* cnt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += gridDim.x * blockDim.x) {
    const Pair p = pairs[i];
    uint32_t a = 0, b = 0;
    if (p.t1 > p.t0) {
      a = lower_bound_tt(tag_c, ts_c, n, p.tag, p.t0);
      b = lower_bound_tt(tag_c, ts_c, n, p.tag, p.t1);
    }
    lo[i] = a;
    cnt[i] = b > a ? b - a : 0;
  }
}

// Copy the selected ranges into one input array: pair i's rows go to
// [out_off[i], out_off[i] + cnt[i]).  A block copies 2048 consecutive output
// rows (row r0 + t + 256 k by thread t): one thread finds the pair of the
// block's first row by binary search, and each thread steps forward from it
// (a block spans few pairs), so the copies are coalesced on both sides.
constexpr uint32_t kGatherRows = 2048;

__global__ void __launch_bounds__(256)
    k_gather(const int32_t* __restrict__ src_c, const int32_t* __restrict__ dst_c,
             const uint32_t* __restrict__ lo, const uint32_t* __restrict__ cnt,
             const uint64_t* __restrict__ out_off, uint32_t npairs, uint64_t total,
             int32_t* __restrict__ src, int32_t* __restrict__ dst) {
  __shared__ uint32_t s_pair;
  for (uint64_t r0 = (uint64_t)blockIdx.x * kGatherRows; r0 < total;
       r0 += (uint64_t)gridDim.x * kGatherRows) {
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t a = 0, b = npairs;  // last pair with out_off <= r0
      while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (out_off[mid] <= r0) a = mid;
        else b = mid;
      }
      s_pair = a;
    }
    __syncthreads();
    uint32_t pi = s_pair;
    const uint64_t r1 = min(r0 + kGatherRows, total);
    for (uint64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      while (pi + 1 < npairs && out_off[pi + 1] <= r) ++pi;
      const uint64_t k = r - out_off[pi];
      if (k >= cnt[pi]) continue;  // alignment gap after a segment
      const uint64_t q = lo[pi] + k;
      src[r] = src_c[q];
      dst[r] = dst_c[q];
    }
  }
}

// ------------------------------------------------------ segmented top-k ---
// The largest-degree nodes of every graph of a wave, in both directions, in
// one set of launches.  Task t = 2 * segment + direction.  As for a single
// graph, each node has the key (degree << 32) | (0xFFFFFFFF - index), and the
// k-th largest key of a task is found by an MSD radix select over 8-bit
// digits; node tiles of all segments share each launch.  V is read from the
// control blocks, so the launches can be recorded before V is known.
constexpr uint32_t kTopkTile = 4096;  // nodes per tile

struct TopkTask {
  uint64_t prefix;     // digits of the k-th key fixed so far
  uint32_t remaining;  // rank of the k-th key among keys matching prefix
  uint32_t count;      // gathered keys
  uint32_t keff;       // min(k, V)
  uint32_t pad[3];
  uint32_t hist[kRadix];
};

// tile map of the node arrays and each task's k; one block
__global__ void k_topk_init(const Ctl* __restrict__ ctls, uint32_t nseg, uint32_t k,
                            uint32_t* tile_start, TopkTask* tasks) {
  __shared__ uint32_t s_sw[33];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nseg; b0 += blockDim.x) {
    const uint32_t sidx = b0 + threadIdx.x;
    uint32_t t = 0, V = 0;
    if (sidx < nseg) {
      V = ctls[sidx].V;
      t = (V + kTopkTile - 1) / kTopkTile;
    }
    uint32_t tot;
    const uint32_t e = block_exclusive_sum<1024>(t, s_sw, tot);
    if (sidx < nseg) {
      tile_start[sidx] = carry + e;
      const uint32_t ke = k < V ? k : V;
      for (int d = 0; d < 2; ++d) {
        tasks[2 * sidx + d].remaining = ke;
        tasks[2 * sidx + d].keff = ke;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_start[nseg] = carry;
}

__device__ __forceinline__ uint64_t node_key(const int64_t* __restrict__ off, uint32_t r) {
  const uint64_t d = (uint64_t)(off[r + 1] - off[r]);
  return (d << 32) | (0xFFFFFFFFu - r);
}

__global__ void __launch_bounds__(256)
    k_topk_hist_seg(const Ctl* __restrict__ ctls, SegMap tiles, TopkTask* tasks, int round) {
  __shared__ uint32_t h[2][kRadix];
  const uint32_t total = __ldg(tiles.start + tiles.nseg);
  const int sh = 56 - 8 * round;
  const uint64_t hi_mask = round == 0 ? 0ull : (~0ull << (64 - 8 * round));
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
    for (int i = threadIdx.x; i < 2 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t sidx = seg_of(tiles, g);
    const Ctl* c = ctls + sidx;
    const uint32_t V = c->V;
    const uint32_t r0 = (g - __ldg(tiles.start + sidx)) * kTopkTile;
    const uint32_t r1 = min(r0 + kTopkTile, V);
    TopkTask* t = tasks + 2 * sidx;
    for (int d = 0; d < 2; ++d) {
      const int64_t* __restrict__ off = d ? c->in_off : c->out_off;
      const uint64_t pre = t[d].prefix;
      if (t[d].keff == 0) continue;
      for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const uint64_t key = node_key(off, r);
        if ((key & hi_mask) == pre) atomicAdd(&h[d][(key >> sh) & 0xFF], 1u);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kRadix; i += blockDim.x) {
      const uint32_t v = (&h[0][0])[i];
      if (v) atomicAdd(&t[i / kRadix].hist[i % kRadix], v);
    }
    __syncthreads();
  }
}

// one warp per task: the digit holding the k-th key, then clear the histogram
__global__ void k_topk_pick_seg(TopkTask* tasks, uint32_t ntasks, int round) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ntasks) return;
  TopkTask* t = tasks + w;
  if (t->keff == 0) return;
  if (lane == 0) {
    const int sh = 56 - 8 * round;
    uint32_t rem = t->remaining;
    for (int d = kRadix - 1; d >= 0; --d) {
      const uint32_t c = t->hist[d];
      if (rem <= c) {
        t->prefix |= (uint64_t)d << sh;
        break;
      }
      rem -= c;
    }
    t->remaining = rem;
  }
  __syncwarp();
  for (int d = lane; d < kRadix; d += 32) t->hist[d] = 0;
}

__global__ void __launch_bounds__(256)
    k_topk_gather_seg(const Ctl* __restrict__ ctls, SegMap tiles, TopkTask* tasks,
                      uint64_t* cand, uint32_t k) {
  const uint32_t total = __ldg(tiles.start + tiles.nseg);
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
    const uint32_t sidx = seg_of(tiles, g);
    const Ctl* c = ctls + sidx;
    const uint32_t V = c->V;
    const uint32_t r0 = (g - __ldg(tiles.start + sidx)) * kTopkTile;
    const uint32_t r1 = min(r0 + kTopkTile, V);
    for (int d = 0; d < 2; ++d) {
      TopkTask* t = tasks + 2 * sidx + d;
      const uint32_t keff = t->keff;
      if (keff == 0) continue;
      const int64_t* __restrict__ off = d ? c->in_off : c->out_off;
      const uint64_t thr = t->prefix;  // the k-th largest key; keys are distinct
      for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const uint64_t key = node_key(off, r);
        if (key >= thr) {
          const uint32_t slot = atomicAdd(&t->count, 1u);
          if (slot < keff) cand[(uint64_t)(2 * sidx + d) * k + slot] = key;
        }
      }
    }
  }
}

// one block per task: bitonic sort of its keff candidates, descending
__global__ void __launch_bounds__(512)
    k_topk_sort_seg(const Ctl* __restrict__ ctls, const TopkTask* __restrict__ tasks,
                    const uint64_t* __restrict__ cand, uint32_t k, int32_t* ids, int64_t* degs) {
  extern __shared__ uint64_t s_keys[];
  const uint32_t task = blockIdx.x;
  const uint32_t n = tasks[task].keff;
  if (n == 0) return;
  const int32_t* __restrict__ node_ids = ctls[task >> 1].node_ids;
  uint32_t p2 = 1;
  while (p2 < n) p2 <<= 1;
  const uint64_t* in = cand + (uint64_t)task * k;
  for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) s_keys[i] = i < n ? in[i] : 0;
  __syncthreads();
  for (uint32_t size = 2; size <= p2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) {
        const uint32_t j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const uint64_t a = s_keys[i], b = s_keys[j];
          if (desc ? (a < b) : (a > b)) {
            s_keys[i] = b;
            s_keys[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const uint64_t key = s_keys[i];
    const uint32_t r = 0xFFFFFFFFu - (uint32_t)key;
    ids[(uint64_t)task * k + i] = node_ids[r];
    degs[(uint64_t)task * k + i] = (int64_t)(key >> 32);
  }
}

uint32_t persistent_blocks(uint32_t per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (uint32_t)sms * per_sm;
}

uint32_t grid_for(uint64_t n, uint32_t per_block, uint32_t cap = 8192) {
  uint64_t g = (n + per_block - 1) / per_block;
  if (g == 0) g = 1;
  return (uint32_t)(g < cap ? g : cap);
}

}  // namespace

// ------------------------------------------------------------ handles --------
struct ringo_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<SegResult> res;
  std::vector<uint32_t> rows;
  std::vector<int32_t*> node_ids, out_nbr, in_nbr;
  std::vector<int64_t*> out_off, in_off;
  std::vector<void*> blocks;  // output blocks of the waves
};

namespace {

// Sort-only run of one segment: the out-sort of (a, b) columns (histogram,
// 4 passes, the rank step, 4 passes); the keys end in ctl->out_sort.result.
struct SoloSort {
  char* zero = nullptr;
  char* scratch = nullptr;
  Ctl* dctl = nullptr;
};

int solo_sort(const int32_t* a, const int32_t* b, uint32_t n, cudaStream_t s, SoloSort* out) {
  const SegLayout L = seg_layout(n);
  const uint64_t zbytes = L.z_total;
  const uint64_t sbytes = L.s_total + al(sizeof(Ctl)) + al(sizeof(SegDesc));
  char* z = (char*)pool_alloc(zbytes, s);
  char* sc = (char*)pool_alloc(sbytes, s);
  if (!z || !sc) {
    pool_free(z, s);
    pool_free(sc, s);
    return RINGO_ENOMEM;
  }
  Ctl* dctl = (Ctl*)(sc + L.s_total);
  SegDesc* ddesc = (SegDesc*)(sc + L.s_total + al(sizeof(Ctl)));
  SegDesc hd{n, a, b, z, sc, nullptr};
  cudaMemsetAsync(z, 0, zbytes, s);
  cudaMemcpyAsync(ddesc, &hd, sizeof(hd), cudaMemcpyHostToDevice, s);
  k_init_ctls<<<1, 256, 0, s>>>(dctl, ddesc);
  // a single segment: its own maps and counters (set on the device)
  out->zero = z;
  out->scratch = sc;
  out->dctl = dctl;
  Ctl* h = (Ctl*)pinned_get(sizeof(Ctl));
  if (!h) return RINGO_ENOMEM;
  memset(h, 0, sizeof(Ctl));
  Launch run = solo_launch(dctl, h, n);
  run.opts = sort_opts_for(0, n);
  cudaMemcpyAsync(&dctl->solo_rows[0], &h->solo_rows[0], 2 * sizeof(uint32_t),
                  cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);  // the staging copy is done before the buffer is reused
  pinned_put(h);
  return enqueue_sort_only(run, s);
}

void solo_sort_free(SoloSort& ss, cudaStream_t s) {
  pool_free(ss.zero, s);
  pool_free(ss.scratch, s);
  ss = SoloSort{};
}

}  // namespace

namespace ringo {

int check_preds(const ringo_select* preds, int32_t npred) {
  if (npred < 0 || (npred > 0 && !preds)) return RINGO_EINVAL;
  for (int32_t i = 0; i < npred; ++i)
    if (preds[i].ntags < 0 || (preds[i].ntags > 0 && !preds[i].tags)) return RINGO_EINVAL;
  return RINGO_OK;
}

// One (tag, window) pair per distinct tag of each predicate, in predicate
// order, so the pairs of a predicate are consecutive.
std::vector<Pair> make_pairs(const ringo_select* preds, int32_t npred) {
  std::vector<Pair> pairs;
  std::vector<int32_t> t;
  for (int32_t i = 0; i < npred; ++i) {
    t.assign(preds[i].tags, preds[i].tags + preds[i].ntags);
    std::sort(t.begin(), t.end());
    t.erase(std::unique(t.begin(), t.end()), t.end());
    for (int32_t tag : t) pairs.push_back(Pair{tag, i, preds[i].t0, preds[i].t1});
  }
  return pairs;
}

int select_ranges(const ringo_base* b, const std::vector<Pair>& pairs, cudaStream_t s, Ranges* r,
                  bool host_lo) {
  const uint32_t np = (uint32_t)pairs.size();
  r->h_cnt.assign(np, 0);
  if (host_lo) r->h_lo.assign(np, 0);
  if (np == 0) return RINGO_OK;
  const size_t bytes = al(sizeof(Pair) * np) + 2 * al(4ull * np);
  char* d = (char*)pool_alloc(bytes, s);
  if (!d) return RINGO_ENOMEM;
  r->block = d;
  Pair* dp = (Pair*)d;
  r->lo = (uint32_t*)(d + al(sizeof(Pair) * np));
  r->cnt = (uint32_t*)(d + al(sizeof(Pair) * np) + al(4ull * np));
  RINGO_CUDA_TRY(cudaMemcpyAsync(dp, pairs.data(), sizeof(Pair) * np, cudaMemcpyHostToDevice, s));
  if (b->n) {
    k_select<<<grid_for(np, 256), 256, 0, s>>>(b->tag_c, b->ts_c, b->n, dp, np, r->lo, r->cnt);
  } else {
    RINGO_CUDA_TRY(cudaMemsetAsync(r->cnt, 0, 4ull * np, s));
  }
  RINGO_CUDA_TRY(cudaMemcpyAsync(r->h_cnt.data(), r->cnt, 4ull * np, cudaMemcpyDeviceToHost, s));
  if (host_lo && b->n)
    RINGO_CUDA_TRY(cudaMemcpyAsync(r->h_lo.data(), r->lo, 4ull * np, cudaMemcpyDeviceToHost, s));
  RINGO_CUDA_TRY(cudaStreamSynchronize(s));
  return RINGO_OK;
}

// Converts the segments of one wave: segment j holds the pairs [first[j],
// first[j + 1]) of the device range arrays lo/cnt (host copy h_cnt).  The
// gather, the whole pipeline and (topk > 0) the segmented top-k of both
// directions are recorded as one CUDA graph and launched once on s.
int run_wave(const ringo_base* b, const uint32_t* d_lo, const uint32_t* d_cnt,
             const uint32_t* h_lo, const uint32_t* h_cnt, const std::vector<size_t>& first,
             uint32_t nseg, uint32_t topk, cudaStream_t s, WaveResult* out) {
  out->seg.assign(nseg, WaveSeg{});
  if (nseg == 0) return RINGO_OK;
  prepare_launches();
  const uint64_t npw = first[nseg];
  std::vector<uint64_t> seg_rows(nseg, 0);
  for (uint32_t k = 0; k < nseg; ++k)
    for (size_t pi = first[k]; pi < first[k + 1]; ++pi) seg_rows[k] += h_cnt[pi];
  std::vector<SegDesc> desc(nseg);
  std::vector<uint32_t> row_start(nseg + 1, 0);
  uint64_t zb = 0, sb = 0, ob = 0, in_rows = 0;
  std::vector<uint64_t> zoff(nseg), soff(nseg), ooff(nseg), ioff(nseg);
  for (uint32_t k = 0; k < nseg; ++k) {
    const uint32_t n = (uint32_t)seg_rows[k];
    const SegLayout L = seg_layout(n);
    zoff[k] = zb; zb += L.z_total;
    soff[k] = sb; sb += L.s_total;
    ooff[k] = ob; ob += L.o_total;
    ioff[k] = in_rows; in_rows += up4(n);
    row_start[k + 1] = row_start[k] + (n ? L.tiles : 0);
  }
  const uint32_t ntasks = topk ? 2 * nseg : 0;
  // after the segments' regions: what must start at zero (claim counters,
  // top-k tasks), then what is written before use (the uploaded row map,
  // maps computed on the device, results)
  const uint64_t zmeta = al(4ull * kNumCounters) + al(sizeof(TopkTask) * ntasks);
  const uint64_t meta = zmeta + al(4ull * (nseg + 1)) * 4 + al(sizeof(SegResult) * nseg);
  const uint64_t tk_bytes = (uint64_t)ntasks * topk;
  char* zr = (char*)pool_alloc(zb + meta, s);
  const bool up_ranges = d_lo == nullptr;  // ranges come from the host
  char* sr = (char*)pool_alloc(sb + al(sizeof(Ctl) * nseg) + al(sizeof(SegDesc) * nseg) +
                                   al(8 * (npw + 1)) + al(8 * in_rows) + al(8 * tk_bytes) +
                                   (up_ranges ? 2 * al(4 * (npw + 1)) : 0),
                               s);
  char* orr = (char*)pool_alloc(ob + al(4 * tk_bytes) + al(8 * tk_bytes), s);
  const size_t hbytes = sizeof(SegResult) * nseg + 12 * tk_bytes + 16;
  char* hbuf = (char*)pinned_get(hbytes);
  out->block = orr;
  if (!zr || !sr || !orr || !hbuf) {
    pool_free(zr, s);
    pool_free(sr, s);
    if (hbuf) pinned_put(hbuf);
    return RINGO_ENOMEM;
  }
  SegResult* hres = (SegResult*)hbuf;
  char* zp = zr + zb;
  uint32_t* d_counters = (uint32_t*)zp;
  TopkTask* d_tasks = (TopkTask*)(zp + al(4ull * kNumCounters));
  char* mp = zp + zmeta;  // not cleared
  uint32_t* d_rows = (uint32_t*)mp;
  uint32_t* d_merge = (uint32_t*)(mp + al(4ull * (nseg + 1)));
  uint32_t* d_blocks = (uint32_t*)(mp + 2 * al(4ull * (nseg + 1)));
  uint32_t* d_ttiles = (uint32_t*)(mp + 3 * al(4ull * (nseg + 1)));
  SegResult* d_res = (SegResult*)(mp + 4 * al(4ull * (nseg + 1)));
  Ctl* d_ctls = (Ctl*)(sr + sb);
  SegDesc* d_desc = (SegDesc*)(sr + sb + al(sizeof(Ctl) * nseg));
  uint64_t* d_pairoff = (uint64_t*)((char*)d_desc + al(sizeof(SegDesc) * nseg));
  int32_t* in_src = (int32_t*)((char*)d_pairoff + al(8 * (npw + 1)));
  int32_t* in_dst = in_src + in_rows;  // two int32 halves of the 8 * in_rows bytes
  uint64_t* d_cand = (uint64_t*)((char*)in_src + al(8 * in_rows));
  if (up_ranges) {
    char* rp = (char*)d_cand + al(8 * tk_bytes);
    d_lo = (const uint32_t*)rp;
    d_cnt = (const uint32_t*)(rp + al(4 * (npw + 1)));
  }
  int32_t* d_tk_ids = (int32_t*)(orr + ob);
  int64_t* d_tk_degs = (int64_t*)(orr + ob + al(4 * tk_bytes));
  // per-pair output offsets inside the wave's input columns
  std::vector<uint64_t> pair_off(npw + 1, 0);
  for (uint32_t k = 0; k < nseg; ++k) {
    uint64_t o = ioff[k];
    for (size_t pi = first[k]; pi < first[k + 1]; ++pi) {
      pair_off[pi] = o;
      o += h_cnt[pi];
    }
  }
  pair_off[npw] = in_rows;
  for (uint32_t k = 0; k < nseg; ++k) {
    desc[k].n = (uint32_t)seg_rows[k];
    desc[k].src = in_src + ioff[k];
    desc[k].dst = in_dst + ioff[k];
    desc[k].zbase = zr + zoff[k];
    desc[k].sbase = sr + soff[k];
    desc[k].obase = orr + ooff[k];
  }
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
  {
    // small host data goes up first, outside the graph
    HostScope hs("host:wave_upload");
    ok = ok && cudaMemcpyAsync(d_desc, desc.data(), sizeof(SegDesc) * nseg,
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d_rows, row_start.data(), 4ull * (nseg + 1),
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d_pairoff, pair_off.data(), 8 * (npw + 1),
                               cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (up_ranges && npw) {
      ok = ok && cudaMemcpyAsync(const_cast<uint32_t*>(d_lo), h_lo, 4 * npw,
                                 cudaMemcpyHostToDevice, s) == cudaSuccess;
      ok = ok && cudaMemcpyAsync(const_cast<uint32_t*>(d_cnt), h_cnt, 4 * npw,
                                 cudaMemcpyHostToDevice, s) == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  }
  Launch L;
  L.ctls = d_ctls;
  L.nseg = nseg;
  L.rows = SegMap{d_rows, nseg};
  L.merge = SegMap{d_merge, nseg};
  L.blocks = SegMap{d_blocks, nseg};
  L.row_slots = row_start[nseg];
  L.counters = d_counters;
  L.opts = sort_opts_for(1, in_rows / nseg);
  int prc = RINGO_OK;
  HostScope* cap_scope = new HostScope("host:wave_capture");
  if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaMemsetAsync(zr, 0, zb + zmeta, cs);
    if (npw)
      k_gather<<<grid_for(in_rows, kGatherRows), 256, 0, cs>>>(b->src_c, b->dst_c, d_lo, d_cnt,
                                                           d_pairoff, (uint32_t)npw, in_rows,
                                                           in_src, in_dst);
    k_init_ctls<<<nseg, 256, 0, cs>>>(d_ctls, d_desc);
    prc = enqueue_phase1(L, cs);
    if (prc == RINGO_OK) prc = enqueue_phase2(L, cs);
    if (prc == RINGO_OK) prc = enqueue_phase3(L, cs);
    if (prc == RINGO_OK && topk) {
      const SegMap tiles{d_ttiles, nseg};
      const uint32_t grid = persistent_blocks(8);
      k_topk_init<<<1, 1024, 0, cs>>>(d_ctls, nseg, topk, d_ttiles, d_tasks);
      for (int round = 0; round < 8; ++round) {
        k_topk_hist_seg<<<grid, 256, 0, cs>>>(d_ctls, tiles, d_tasks, round);
        k_topk_pick_seg<<<(ntasks + 7) / 8, 256, 0, cs>>>(d_tasks, ntasks, round);
      }
      k_topk_gather_seg<<<grid, 256, 0, cs>>>(d_ctls, tiles, d_tasks, d_cand, topk);
      uint32_t p2 = 1;
      while (p2 < topk) p2 <<= 1;
      k_topk_sort_seg<<<ntasks, 512, 8 * p2, cs>>>(d_ctls, d_tasks, d_cand, topk, d_tk_ids,
                                                   d_tk_degs);
      if (cudaGetLastError() != cudaSuccess) prc = RINGO_ECUDA;
    }
    k_collect<<<grid_for(nseg, 256), 256, 0, cs>>>(d_ctls, nseg, d_res);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    ok = prc == RINGO_OK && ce == cudaSuccess;
  }
  delete cap_scope;
  {
    HostScope hs("host:wave_instantiate");
    ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  }
  HostScope* run_scope = new HostScope("host:wave_run");
  {
    ProfScope ps("batch_wave", s);
    ok = ok && cudaGraphLaunch(exec, s) == cudaSuccess;
  }
  ok = ok && cudaMemcpyAsync(hres, d_res, sizeof(SegResult) * nseg, cudaMemcpyDeviceToHost,
                             s) == cudaSuccess;
  int32_t* h_tk_ids = (int32_t*)(hbuf + sizeof(SegResult) * nseg);
  int64_t* h_tk_degs = (int64_t*)(hbuf + ((sizeof(SegResult) * nseg + 4 * tk_bytes + 7) & ~7ull));
  if (tk_bytes) {
    ok = ok && cudaMemcpyAsync(h_tk_ids, d_tk_ids, 4 * tk_bytes, cudaMemcpyDeviceToHost, s) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_tk_degs, d_tk_degs, 8 * tk_bytes, cudaMemcpyDeviceToHost, s) ==
                   cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  delete run_scope;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  int rc = RINGO_OK;
  if (!ok) {
    set_error(std::string("wave: CUDA error: ") + cudaGetErrorString(cudaGetLastError()));
    rc = prc != RINGO_OK ? prc : RINGO_ECUDA;
  } else {
    for (uint32_t k = 0; k < nseg; ++k) {
      WaveSeg& g = out->seg[k];
      g.res = hres[k];
      g.res_rows = desc[k].n;
      if (g.res.err) {
        set_error("wave: a bounded device wait expired");
        rc = (g.res.err & kErrRemap) ? RINGO_ECUDA : RINGO_ETIMEOUT;
      }
      const SegLayout Lk = seg_layout(desc[k].n);
      char* o = desc[k].obase;
      g.node_ids = (int32_t*)(o + Lk.node_ids);
      g.out_off = (int64_t*)(o + Lk.out_off);
      g.out_nbr = (int32_t*)(o + Lk.out_nbr);
      g.in_off = (int64_t*)(o + Lk.in_off);
      g.in_nbr = (int32_t*)(o + Lk.in_nbr);
      if (desc[k].n == 0) {  // empty selection: offsets {0}
        cudaMemsetAsync(g.out_off, 0, 8, s);
        cudaMemsetAsync(g.in_off, 0, 8, s);
      }
    }
    if (tk_bytes) {
      out->topk_ids.assign(h_tk_ids, h_tk_ids + tk_bytes);
      out->topk_degs.assign(h_tk_degs, h_tk_degs + tk_bytes);
    }
  }
  pinned_put(hbuf);
  pool_free(zr, s);
  pool_free(sr, s);
  return rc;
}

// ------------------------------------------------------------- tuning -----
// Wave size: the rows converted by one captured launch.  Outputs of every
// wave stay allocated (about 48 B per selected row, sized for V <= 2n); a
// wave's scratch and gathered input take about 50 B per row on top.  The
// default is the largest wave that fits in 85% of the available device
// memory; ringo_batch_autotune times candidates on a real predicate set and
// records the choice per (GPU, size class of the mean selection), tune.cu.

int64_t fit_wave_rows(uint64_t total_rows) {
  const double usable = 0.85 * (double)pool_available();
  double w = (usable - 48.0 * (double)total_rows) / 50.0;
  const double lo = 16.0 * (1 << 20);
  if (w < lo) w = lo;
  if (w > (double)total_rows) w = (double)total_rows;
  return std::max<int64_t>(1, (int64_t)w);
}

int64_t choose_wave_rows(int32_t npred, uint64_t total_rows) {
  const int64_t fit = fit_wave_rows(total_rows);
  const int64_t tuned = tuned_wave_rows(npred > 0 ? total_rows / (uint64_t)npred : 0);
  return tuned > 0 ? std::min(tuned, fit) : fit;
}

uint64_t wave_seg_bytes(uint32_t n, uint32_t topk) {
  const SegLayout L = seg_layout(n);
  return L.z_total + L.s_total + L.o_total + 8 * up4(n) + al(sizeof(Ctl)) + sizeof(SegDesc) +
         sizeof(SegResult) + 2 * sizeof(TopkTask) + 40ull * topk + 4096;
}

uint64_t wave_seg_output_bytes(uint32_t n) { return seg_layout(n).o_total; }

}  // namespace ringo

extern "C" {

int ringo_base_table_load(const int32_t* src, const int32_t* dst, const int64_t* ts,
                          const int32_t* tag, int64_t nrows, void* stream, ringo_base** out) {
  if (!out) return RINGO_EINVAL;
  *out = nullptr;
  if (nrows < 0 || (nrows > 0 && (!src || !dst || !ts || !tag))) {
    set_error("ringo_base_table_load: nrows < 0 or NULL column");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF) {
    set_error("ringo_base_table_load: nrows exceeds 2^31 - 1");
    return RINGO_ERANGE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ringo_base* b = new ringo_base();
  cudaGetDevice(&b->device);
  const uint32_t n = (uint32_t)nrows;
  b->n = n;
  if (n == 0) {
    *out = b;
    return RINGO_OK;
  }
  int rc = RINGO_OK;
  b->src_c = (int32_t*)pool_alloc(4ull * n, s);
  b->dst_c = (int32_t*)pool_alloc(4ull * n, s);
  b->ts_c = (int64_t*)pool_alloc(8ull * n, s);
  b->tag_c = (int32_t*)pool_alloc(4ull * n, s);
  char* tmp = (char*)pool_alloc(al(16) + 3 * al(4ull * n) + al(4ull * n), s);
  long long hmm[2] = {0, 0};
  SoloSort s1, s2;
  if (!b->src_c || !b->dst_c || !b->ts_c || !b->tag_c || !tmp) {
    rc = RINGO_ENOMEM;
  } else {
    long long* mm = (long long*)tmp;
    int32_t* ca = (int32_t*)(tmp + al(16));
    int32_t* cb = (int32_t*)(tmp + al(16) + al(4ull * n));
    int32_t* o1 = (int32_t*)(tmp + al(16) + 2 * al(4ull * n));
    const long long init[2] = {LLONG_MAX, LLONG_MIN};
    cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s);
    k_minmax_i64<<<grid_for(n, 256, 2048), 256, 0, s>>>(ts, n, mm);
    cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      rc = RINGO_ECUDA;
    } else if ((unsigned long long)hmm[1] - (unsigned long long)hmm[0] >= (1ull << 32)) {
      set_error("ringo_base_table_load: the ts range must be below 2^32");
      rc = RINGO_ERANGE;
    } else {
      k_stage1_cols<<<grid_for(n, 256), 256, 0, s>>>(ts, mm, n, ca, cb);
      rc = solo_sort(ca, cb, n, s, &s1);
      if (rc == RINGO_OK) {
        k_stage2_cols<<<grid_for(n, 256), 256, 0, s>>>(s1.dctl, tag, n, ca, cb, o1);
        rc = solo_sort(ca, cb, n, s, &s2);
      }
      if (rc == RINGO_OK) {
        k_cluster_gather<<<grid_for(n, 256), 256, 0, s>>>(s2.dctl, o1, n, src, dst, ts, tag,
                                                          b->src_c, b->dst_c, b->ts_c, b->tag_c);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
          set_error("ringo_base_table_load: CUDA error");
          rc = RINGO_ECUDA;
        }
      }
    }
  }
  solo_sort_free(s1, s);
  solo_sort_free(s2, s);
  pool_free(tmp, s);
  if (rc != RINGO_OK) {
    pool_free(b->src_c, s);
    pool_free(b->dst_c, s);
    pool_free(b->ts_c, s);
    pool_free(b->tag_c, s);
    cudaStreamSynchronize(s);
    delete b;
    return rc;
  }
  *out = b;
  return RINGO_OK;
}

int ringo_base_table_rows(const ringo_base* b, int64_t* nrows) {
  if (!b || !nrows) return RINGO_EINVAL;
  *nrows = b->n;
  return RINGO_OK;
}

void ringo_base_table_free(ringo_base* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  pool_free(b->src_c, nullptr);
  pool_free(b->dst_c, nullptr);
  pool_free(b->ts_c, nullptr);
  pool_free(b->tag_c, nullptr);
  cudaStreamSynchronize(nullptr);
  delete b;
}

int ringo_select_count(const ringo_base* b, const ringo_select* preds, int32_t npred,
                       void* stream, int64_t* counts) {
  if (!b || (npred > 0 && !counts)) return RINGO_EINVAL;
  if (int rc = check_preds(preds, npred)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<Pair> pairs = make_pairs(preds, npred);
  Ranges rg;
  int rc = select_ranges(b, pairs, s, &rg);
  pool_free(rg.block, s);
  if (rc != RINGO_OK) return rc;
  for (int32_t i = 0; i < npred; ++i) counts[i] = 0;
  for (size_t i = 0; i < pairs.size(); ++i) counts[pairs[i].seg] += rg.h_cnt[i];
  return RINGO_OK;
}

int ringo_select_gather(const ringo_base* b, const ringo_select* pred, int32_t* d_src,
                        int32_t* d_dst, int64_t cap, int64_t* n, void* stream) {
  if (!b || !pred || !n) return RINGO_EINVAL;
  if (int rc = check_preds(pred, 1)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const std::vector<Pair> pairs = make_pairs(pred, 1);
  Ranges rg;
  int rc = select_ranges(b, pairs, s, &rg);
  if (rc != RINGO_OK) {
    pool_free(rg.block, s);
    return rc;
  }
  uint64_t total = 0;
  std::vector<uint64_t> off(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) {
    off[i] = total;
    total += rg.h_cnt[i];
  }
  *n = (int64_t)total;
  if ((int64_t)total > cap || (total && (!d_src || !d_dst))) {
    pool_free(rg.block, s);
    set_error("ringo_select_gather: selection larger than cap");
    return RINGO_ERANGE;
  }
  if (total) {
    uint64_t* doff = (uint64_t*)pool_alloc(8 * off.size(), s);
    if (!doff) {
      pool_free(rg.block, s);
      return RINGO_ENOMEM;
    }
    cudaMemcpyAsync(doff, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, s);
    k_gather<<<grid_for(total, kGatherRows), 256, 0, s>>>(b->src_c, b->dst_c, rg.lo, rg.cnt, doff,
                                                      (uint32_t)pairs.size(), total, d_src, d_dst);
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    pool_free(doff, s);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      pool_free(rg.block, s);
      set_error("ringo_select_gather: CUDA error");
      return RINGO_ECUDA;
    }
  }
  pool_free(rg.block, s);
  return RINGO_OK;
}

int ringo_convert_batch(const ringo_base* b, const ringo_select* preds, int32_t npred,
                        int64_t wave_rows, void* stream, ringo_batch** out) {
  if (!b || !out) return RINGO_EINVAL;
  *out = nullptr;
  if (int rc = check_preds(preds, npred)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ringo_batch* bt = new ringo_batch();
  cudaGetDevice(&bt->device);
  bt->stream = s;
  bt->res.assign(npred, SegResult{});
  bt->rows.assign(npred, 0);
  bt->node_ids.assign(npred, nullptr);
  bt->out_nbr.assign(npred, nullptr);
  bt->in_nbr.assign(npred, nullptr);
  bt->out_off.assign(npred, nullptr);
  bt->in_off.assign(npred, nullptr);
  const std::vector<Pair> pairs = make_pairs(preds, npred);
  Ranges rg;
  int rc = select_ranges(b, pairs, s, &rg);
  // pairs of predicate i: [first[i], first[i + 1])
  std::vector<size_t> first(npred + 1, 0);
  std::vector<uint64_t> seg_rows(npred, 0);
  for (size_t i = 0; i < pairs.size(); ++i) {
    seg_rows[pairs[i].seg] += rg.h_cnt[i];
    first[pairs[i].seg + 1] = i + 1;
  }
  for (int32_t i = 0; i < npred; ++i) first[i + 1] = std::max(first[i + 1], first[i]);
  for (int32_t i = 0; rc == RINGO_OK && i < npred; ++i)
    if (seg_rows[i] > 0x7FFFFFFFull) {
      set_error("ringo_convert_batch: a selection exceeds 2^31 - 1 rows");
      rc = RINGO_ERANGE;
    }
  if (wave_rows <= 0) {
    uint64_t total = 0;
    for (uint64_t r : seg_rows) total += r;
    wave_rows = choose_wave_rows(npred, total);
  }
  int32_t a = 0;
  while (rc == RINGO_OK && a < npred) {
    // predicates [a, z) form a wave (empty selections ride along for free)
    int32_t z = a;
    uint64_t rows = 0;
    while (z < npred && (z == a || rows + seg_rows[z] <= (uint64_t)wave_rows)) rows += seg_rows[z++];
    std::vector<size_t> wf(z - a + 1);
    for (int32_t k = a; k <= z; ++k) wf[k - a] = first[k] - first[a];
    WaveResult w;
    rc = run_wave(b, rg.lo + first[a], rg.cnt + first[a], nullptr, rg.h_cnt.data() + first[a], wf,
                  (uint32_t)(z - a), 0, s, &w);
    if (w.block) bt->blocks.push_back(w.block);
    if (rc != RINGO_OK) break;
    for (int32_t k = 0; k < z - a; ++k) {
      const WaveSeg& g = w.seg[k];
      bt->res[a + k] = g.res;
      bt->rows[a + k] = g.res_rows;
      bt->node_ids[a + k] = g.node_ids;
      bt->out_off[a + k] = g.out_off;
      bt->out_nbr[a + k] = g.out_nbr;
      bt->in_off[a + k] = g.in_off;
      bt->in_nbr[a + k] = g.in_nbr;
    }
    a = z;
  }
  cudaStreamSynchronize(s);
  pool_free(rg.block, s);
  if (rc != RINGO_OK) {
    ringo_batch_free(bt);
    return rc;
  }
  *out = bt;
  return RINGO_OK;
}

int ringo_batch_autotune(const ringo_base* b, const ringo_select* preds, int32_t npred,
                         void* stream, int64_t* best_wave_rows, double* best_ms) {
  if (!b || !best_wave_rows) return RINGO_EINVAL;
  if (int rc = check_preds(preds, npred)) return rc;
  int64_t counts_sum = 0;
  {
    std::vector<int64_t> counts(std::max<int32_t>(npred, 1));
    if (int rc = ringo_select_count(b, preds, npred, stream, counts.data())) return rc;
    for (int32_t i = 0; i < npred; ++i) counts_sum += counts[i];
  }
  const uint64_t total = (uint64_t)counts_sum;
  const int64_t fit = fit_wave_rows(total);
  std::vector<int64_t> cand;
  for (int64_t w = fit; w >= (16ll << 20) && cand.size() < 4; w /= 2) cand.push_back(w);
  if (cand.empty()) cand.push_back(fit);
  int64_t best = cand[0];
  double best_t = 1e300;
  for (size_t i = 0; i <= cand.size(); ++i) {
    const int64_t w = cand[i == 0 ? 0 : i - 1];  // the first candidate runs twice (warm-up)
    const auto t0 = std::chrono::steady_clock::now();
    ringo_batch* bt = nullptr;
    const int rc = ringo_convert_batch(b, preds, npred, w, stream, &bt);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ringo_batch_free(bt);
    if (rc == RINGO_ENOMEM) continue;  // too large for the memory left
    if (rc != RINGO_OK) return rc;
    if (i > 0 && ms < best_t) {
      best_t = ms;
      best = w;
    }
  }
  if (best_t == 1e300) {
    set_error("ringo_batch_autotune: no candidate wave fits in device memory");
    return RINGO_ENOMEM;
  }
  // the pass variants at the chosen wave size (each run once; the variant
  // in use has just run, so the device is warm)
  SweepOpts best_o = sort_opts_for(1, npred > 0 ? total / (uint64_t)npred : 0);
  {
    const ForcedOptsGuard keep;  // candidates are forced one after another
    int rc = RINGO_OK;
    const auto measure = [&](const SweepOpts& so) {
      const ringo_sort_opts o{so.rank_method, so.prefetch_waves, 0, so.in_digit_bits, 0};
      ringo_sort_opts_force(&o);
      const auto t0 = std::chrono::steady_clock::now();
      ringo_batch* bt = nullptr;
      rc = ringo_convert_batch(b, preds, npred, best, stream, &bt);
      const double ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      ringo_batch_free(bt);
      if (rc == RINGO_OK && ms < best_t) {
        best_t = ms;
        best_o = so;
      }
    };
    for_each_candidate(measure, [&] { return best_o; }, [&] { return rc == RINGO_OK; });
    if (rc != RINGO_OK) return rc;
  }
  record_tuned(1, npred > 0 ? total / (uint64_t)npred : 0, best_o, best, best_t, 0, 0);
  *best_wave_rows = best;
  if (best_ms) *best_ms = best_t;
  return RINGO_OK;
}

int ringo_batch_num_graphs(const ringo_batch* bt, int32_t* n) {
  if (!bt || !n) return RINGO_EINVAL;
  *n = (int32_t)bt->res.size();
  return RINGO_OK;
}

int ringo_batch_graph_info(const ringo_batch* bt, int32_t i, ringo_graph_info* info) {
  if (!bt || !info || i < 0 || i >= (int32_t)bt->res.size()) return RINGO_EINVAL;
  const SegResult& r = bt->res[i];
  memset(info, 0, sizeof(*info));
  info->nrows = bt->rows[i];
  info->num_nodes = r.V;
  info->num_edges = r.E;
  info->num_src_nodes = r.Vs;
  info->num_dst_nodes = r.Vd;
  info->out_sort_passes = (int32_t)r.out_passes;
  info->in_sort_passes = (int32_t)r.in_passes;
  return RINGO_OK;
}

int ringo_batch_copy_graph_to_host(const ringo_batch* bt, int32_t i, int32_t* h_node_ids,
                                   int64_t* h_out_off, int32_t* h_out_nbr, int64_t* h_in_off,
                                   int32_t* h_in_nbr) {
  if (!bt || i < 0 || i >= (int32_t)bt->res.size()) return RINGO_EINVAL;
  cudaStream_t s = bt->stream;
  const size_t V = bt->res[i].V, E = bt->res[i].E;
  if (h_node_ids && V)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_node_ids, bt->node_ids[i], 4 * V, cudaMemcpyDeviceToHost, s));
  if (h_out_off)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_out_off, bt->out_off[i], 8 * (V + 1), cudaMemcpyDeviceToHost, s));
  if (h_out_nbr && E)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_out_nbr, bt->out_nbr[i], 4 * E, cudaMemcpyDeviceToHost, s));
  if (h_in_off)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_in_off, bt->in_off[i], 8 * (V + 1), cudaMemcpyDeviceToHost, s));
  if (h_in_nbr && E)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_in_nbr, bt->in_nbr[i], 4 * E, cudaMemcpyDeviceToHost, s));
  RINGO_CUDA_TRY(cudaStreamSynchronize(s));
  return RINGO_OK;
}

int ringo_batch_degree_topk(const ringo_batch* bt, int32_t i, int dir, int32_t k, int32_t* h_ids,
                            int64_t* h_degs, int32_t* n_out) {
  if (!bt || !n_out || i < 0 || i >= (int32_t)bt->res.size() || k < 0 ||
      (dir != RINGO_OUT && dir != RINGO_IN))
    return RINGO_EINVAL;
  if (k > 4096) return RINGO_ERANGE;
  const uint32_t V = bt->res[i].V;
  const uint32_t kk = (uint32_t)k < V ? (uint32_t)k : V;
  *n_out = (int32_t)kk;
  if (kk == 0) return RINGO_OK;
  if (!h_ids || !h_degs) return RINGO_EINVAL;
  cudaStream_t s = bt->stream;
  const size_t sbytes = topk_scratch_bytes(V, kk);
  char* buf = (char*)pool_alloc(al(sbytes) + al(4ull * kk) + 8ull * kk, s);
  if (!buf) return RINGO_ENOMEM;
  int32_t* d_ids = (int32_t*)(buf + al(sbytes));
  int64_t* d_degs = (int64_t*)(buf + al(sbytes) + al(4ull * kk));
  int rc = RINGO_OK;
  if (launch_topk(bt->node_ids[i], dir == RINGO_OUT ? bt->out_off[i] : bt->in_off[i], V, kk,
                  d_ids, d_degs, buf, sbytes, s) != 0)
    rc = RINGO_EINVAL;
  if (rc == RINGO_OK) {
    cudaError_t e = cudaMemcpyAsync(h_ids, d_ids, 4ull * kk, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_degs, d_degs, 8ull * kk, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = RINGO_ECUDA;
  }
  pool_free(buf, s);
  return rc;
}

int ringo_batch_graph_to_edge_table(const ringo_batch* bt, int32_t i, int dir, int32_t* d_src,
                                    int32_t* d_dst, int64_t cap, int64_t* n, void* stream) {
  if (!bt || !n || i < 0 || i >= (int32_t)bt->res.size() || cap < 0 ||
      (dir != RINGO_OUT && dir != RINGO_IN))
    return RINGO_EINVAL;
  const int64_t E = bt->res[i].E;
  *n = E;
  if (E > cap) return RINGO_ERANGE;
  if (E && (!d_src || !d_dst)) return RINGO_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : bt->stream;
  const uint32_t V = bt->res[i].V;
  if (dir == RINGO_OUT)
    return launch_edge_table(bt->node_ids[i], bt->out_off[i], bt->out_nbr[i], V, (uint64_t)E,
                             d_src, d_dst, s);
  return launch_edge_table(bt->node_ids[i], bt->in_off[i], bt->in_nbr[i], V, (uint64_t)E, d_dst,
                           d_src, s);
}

void ringo_batch_free(ringo_batch* bt) {
  if (!bt) return;
  for (void* p : bt->blocks) pool_free(p, bt->stream);
  cudaStreamSynchronize(bt->stream);
  delete bt;
}

}  // extern "C"
