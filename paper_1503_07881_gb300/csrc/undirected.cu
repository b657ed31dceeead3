// Undirected conversion and triangle counting (ringo_table_to_undirected_graph,
// ringo_graph_count_triangles): the paper's undirected workload (Section 4,
// Table "paralg": triangle counting on the undirected LiveJournal and
// Twitter2010 graphs).
//
// Undirected conversion: each row (s, d) is the edge {s, d}, so a node's
// undirected list is the union of its directed out- and in-lists.  The table
// goes through the directed conversion once; then the two sorted lists of
// every node are merged, an element present in both kept once.  In merged
// position space node v starts at W(v) = out_off[v] + in_off[v]; each block
// takes 2048 consecutive positions, found by a search for the node and a
// merge-path split inside it, so a hub's lists are shared among many blocks
// and many small nodes fill one block.  A counting pass, a scan of the block
// counts and a writing pass give the lists (each block's output staged in
// shared memory and stored contiguously) and the offsets (each node's first
// element is never a duplicate).  Both CSR directions hold the same lists.
//
// Triangles: edges are oriented from the endpoint of smaller (degree, index)
// to the larger, which keeps every oriented list below sqrt(2E) entries; a
// triangle {a, b, c} with a < b < c in that order is counted exactly once, as
// c in both N+(a) and N+(b).  For each oriented edge (u, v), N+(u) and N+(v)
// (both sorted by node index) are merged when their lengths are close, else
// the shorter is searched, element by element, in the longer.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kScanTileNodes = 2048;  // nodes per block of the offset scan

// deg[v], and deg16[v] = min(deg[v], 65535): the order of (degree, index)
// is decided by the 16-bit copy (half the bytes, so the gathers of it stay in
// L2) except between two nodes of degree 65535 or more
constexpr uint32_t kDeg16Max = 0xFFFFu;

__global__ void k_tc_degree(const int64_t* __restrict__ off, uint32_t V, int32_t* __restrict__ deg,
                            uint16_t* __restrict__ deg16) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const int64_t d = off[v + 1] - off[v];
    deg[v] = (int32_t)d;
    deg16[v] = (uint16_t)(d < (int64_t)kDeg16Max ? d : (int64_t)kDeg16Max);
  }
}

// u -> v when (deg u, u) < (deg v, v); self-loops dropped
__device__ __forceinline__ bool oriented(const int32_t* __restrict__ deg,
                                         const uint16_t* __restrict__ deg16, int32_t du,
                                         uint32_t du16, uint32_t u, uint32_t v) {
  if (v == u) return false;
  const uint32_t dv16 = __ldg(deg16 + v);
  if (dv16 != du16) return dv16 > du16;
  if (du16 < kDeg16Max) return v > u;  // the same degree
  const int32_t dv = __ldg(deg + v);
  return dv > du || (dv == du && v > u);
}

// exclusive scan of cnt into off+, in three steps: tile sums, one block over
// the tile sums, each tile scanned from its offset
__global__ void __launch_bounds__(256)
    k_tc_tile_sums(const uint32_t* __restrict__ cnt, uint32_t V, uint64_t* __restrict__ tsum) {
  __shared__ uint64_t s[256];
  const uint32_t base = blockIdx.x * kScanTileNodes;
  uint64_t t = 0;
  for (uint32_t k = threadIdx.x; k < kScanTileNodes && base + k < V; k += blockDim.x) t += cnt[base + k];
  s[threadIdx.x] = t;
  __syncthreads();
  for (uint32_t k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) tsum[blockIdx.x] = s[0];
}

// exclusive scan of tsum[0, tiles) in place, tsum[tiles] = the total; one
// block of 1024 threads, each over a contiguous run of the tile sums
__global__ void __launch_bounds__(1024) k_scan_tile_sums(uint64_t* __restrict__ tsum, uint32_t tiles) {
  __shared__ uint64_t s_sw[1024 / 32 + 1];
  const uint32_t per = (tiles + 1023) / 1024;
  const uint32_t b = threadIdx.x * per;
  const uint32_t e = min(b + per, tiles);
  uint64_t local = 0;
  for (uint32_t t = b; t < e; ++t) local += tsum[t];
  uint64_t total;
  uint64_t run = block_exclusive_sum<1024>(local, s_sw, total);
  for (uint32_t t = b; t < e; ++t) {
    const uint64_t c = tsum[t];
    tsum[t] = run;
    run += c;
  }
  if (threadIdx.x == 0) tsum[tiles] = total;
}

__global__ void __launch_bounds__(256)
    k_tc_tile_scan(const uint32_t* __restrict__ cnt, uint32_t V, const uint64_t* __restrict__ tsum,
                   uint32_t tiles, int64_t* __restrict__ offp) {
  __shared__ uint64_t s_sw[9];
  const uint32_t base = blockIdx.x * kScanTileNodes;
  constexpr uint32_t kPer = kScanTileNodes / 256;  // 8 nodes per thread, in order
  uint32_t c[kPer];
  uint64_t local = 0;
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint32_t v = base + threadIdx.x * kPer + q;
    c[q] = v < V ? cnt[v] : 0u;
    local += c[q];
  }
  uint64_t total;
  uint64_t run = tsum[blockIdx.x] + block_exclusive_sum<256>(local, s_sw, total);
#pragma unroll
  for (uint32_t q = 0; q < kPer; ++q) {
    const uint32_t v = base + threadIdx.x * kPer + q;
    if (v < V) offp[v] = (int64_t)run;
    run += c[q];
  }
  if (blockIdx.x == tiles - 1 && threadIdx.x == 0) offp[V] = (int64_t)tsum[tiles];
}

// oriented lists, each in its node's own slot of the undirected lists (from
// off[u]; ascending index) with its length in cnt[u]: one pass, no scan
__global__ void __launch_bounds__(256)
    k_tc_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ nbr,
              const int32_t* __restrict__ deg, const uint16_t* __restrict__ deg16, uint32_t V,
              uint32_t* __restrict__ cnt, int32_t* __restrict__ nbrp) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < V;
       u += warps) {
    const int64_t a = off[u], b = off[u + 1];
    const int32_t du = deg[u];
    const uint32_t du16 = deg16[u];
    int64_t w = a;
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane;
      const uint32_t v = e < b ? (uint32_t)nbr[e] : 0u;
      const bool keep = e < b && oriented(deg, deg16, du, du16, (uint32_t)u, v);
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) nbrp[w + __popc(m & lt)] = (int32_t)v;
      w += __popc(m);
    }
    if (lane == 0) cnt[u] = (uint32_t)(w - a);
  }
}

// |A ∩ B| for sorted lists.  Lists of similar length (the longer at most
// kTcMergeRatio times the shorter) are merged: one pass over both, in order,
// consecutive loads that mostly hit L1.  A list much shorter than the other
// has each of its elements searched in the longer one (a search per element,
// resumed from the last position).
constexpr uint64_t kTcMergeRatio = 4;
__device__ __forceinline__ uint32_t intersect(const int32_t* __restrict__ a, uint32_t na,
                                              const int32_t* __restrict__ b, uint32_t nb) {
  if (na > nb) {
    const int32_t* t = a;
    a = b;
    b = t;
    const uint32_t tn = na;
    na = nb;
    nb = tn;
  }
  if (na == 0) return 0;
  uint32_t c = 0;
  if ((uint64_t)nb <= (uint64_t)na * kTcMergeRatio) {
    uint32_t i = 0, j = 0;
    int32_t x = a[0], y = b[0];
    while (true) {
      if (x < y) {
        if (++i == na) break;
        x = a[i];
      } else if (x > y) {
        if (++j == nb) break;
        y = b[j];
      } else {
        ++c;
        if (++i == na || ++j == nb) break;
        x = a[i];
        y = b[j];
      }
    }
    return c;
  }
  uint32_t lo0 = 0;
  for (uint32_t i = 0; i < na; ++i) {
    const int32_t x = a[i];
    uint32_t lo = lo0, hi = nb;  // the elements of a ascend: search from the last position
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (b[mid] < x) lo = mid + 1;
      else hi = mid;
    }
    if (lo < nb && b[lo] == x) ++c;
    lo0 = lo;
    if (lo0 >= nb) break;
  }
  return c;
}

// the oriented lists packed in node order: N+(u) moves from its slot
// nbrs[off[u], off[u] + cnt[u]) to nbrp[offp[u], offp[u + 1]) (offp: the
// exclusive scan of cnt), so the lists the intersections read lie together
__global__ void __launch_bounds__(256)
    k_tc_pack(const int64_t* __restrict__ off, const uint32_t* __restrict__ cnt,
              const int32_t* __restrict__ nbrs, const int64_t* __restrict__ offp, uint32_t V,
              int32_t* __restrict__ nbrp) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < V;
       u += warps) {
    const int64_t a = off[u], w = offp[u];
    const uint32_t n = cnt[u];
    for (uint32_t k = lane; k < n; k += 32) nbrp[w + k] = nbrs[a + k];
  }
}

// one warp per node u; lanes over v in N+(u)
__global__ void __launch_bounds__(256)
    k_tc_triangles(const int64_t* __restrict__ offp, const int32_t* __restrict__ nbrp, uint32_t V,
                   unsigned long long* __restrict__ total) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long acc = 0;
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < V;
       u += warps) {
    const int64_t a = offp[u], b = offp[u + 1];
    if (b - a < 2) continue;
    for (int64_t e = a + lane; e < b; e += 32) {
      const uint32_t v = (uint32_t)nbrp[e];
      if (v >= V) continue;
      const int64_t va = offp[v], vb = offp[v + 1];
      acc += intersect(nbrp + a, (uint32_t)(b - a), nbrp + va, (uint32_t)(vb - va));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0 && acc) atomicAdd(total, acc);
}

// ------------------------------------------------------- undirected merge --
constexpr uint32_t kUmThreads = 256;
constexpr uint32_t kUmItems = 8;                       // merged positions per thread
constexpr uint32_t kUmTile = kUmThreads * kUmItems;    // merged positions per block

// The directed graph whose lists are merged; W = 2E merged positions.
struct UmGraph {
  const int64_t* oo;
  const int32_t* on;
  const int64_t* io;
  const int32_t* in;
  uint32_t V;
  uint64_t W;
};

// Where a block's positions start: the node holding the first one, and how
// many of that node's out- (i) and in-elements (j) come before it.
struct UmSplit {
  uint32_t v, i, j, pad;
};

__device__ __forceinline__ uint64_t um_w(const UmGraph& g, uint32_t v) {
  return (uint64_t)(__ldg(g.oo + v) + __ldg(g.io + v));
}

// The largest v in [lo, hi] with W(v) <= p (W(lo) <= p).
__device__ __forceinline__ uint32_t um_node(const UmGraph& g, uint32_t lo, uint32_t hi, uint64_t p) {
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (um_w(g, mid) <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Merge path of sorted A[na], B[nb] with ties to A: how many of the first q
// merged elements come from A.
__device__ __forceinline__ uint32_t um_path(const int32_t* __restrict__ A, uint32_t na,
                                            const int32_t* __restrict__ B, uint32_t nb, uint32_t q) {
  uint32_t lo = q > nb ? q - nb : 0u, hi = q < na ? q : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(A + mid) <= __ldg(B + (q - 1 - mid))) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// part[c] for c in [0, nch]: the split at position min(c * kUmTile, W)
__global__ void __launch_bounds__(256)
    k_um_partition(UmGraph g, uint32_t nch, UmSplit* __restrict__ part) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= nch; c += gridDim.x * blockDim.x) {
    const uint64_t p = (uint64_t)c * kUmTile < g.W ? (uint64_t)c * kUmTile : g.W;
    UmSplit sp{um_node(g, 0, g.V, p), 0, 0, 0};
    if (sp.v < g.V) {
      const int64_t a0 = g.oo[sp.v], b0 = g.io[sp.v];
      const uint32_t na = (uint32_t)(g.oo[sp.v + 1] - a0), nb = (uint32_t)(g.io[sp.v + 1] - b0);
      const uint32_t q = (uint32_t)(p - (uint64_t)(a0 + b0));
      sp.i = um_path(g.on + a0, na, g.in + b0, nb, q);
      sp.j = q - sp.i;
    }
    part[c] = sp;
  }
}

// Block c merges positions [c * kUmTile, min((c + 1) * kUmTile, W)), eight
// consecutive ones per thread: the thread finds its node among the block's
// nodes and its split inside that node, then merges on, into the next node
// when one is used up.  An in-element equal to the last out-element taken in
// the same node is a duplicate (ties go to the out-list first).
//   WRITE = false: cnt[c] = the block's kept elements;
//   WRITE = true: the kept elements to unbr from base[c] on, and uoff[v]
//                 for every node whose first element the block holds.
template <bool WRITE>
__global__ void __launch_bounds__(kUmThreads)
    k_um_merge(UmGraph g, const UmSplit* __restrict__ part, uint32_t* __restrict__ cnt,
               const int64_t* __restrict__ base, int64_t* __restrict__ uoff,
               int32_t* __restrict__ unbr) {
  __shared__ int32_t s_out[WRITE ? kUmTile : 1];
  __shared__ uint32_t s_sw[kUmThreads / 32 + 1];
  const uint32_t c = blockIdx.x;
  const uint64_t p0 = (uint64_t)c * kUmTile;
  const uint64_t pend = p0 + kUmTile < g.W ? p0 + kUmTile : g.W;
  const uint64_t pt = p0 + (uint64_t)threadIdx.x * kUmItems;
  const uint32_t nitems =
      pt >= pend ? 0u : (pend - pt < kUmItems ? (uint32_t)(pend - pt) : kUmItems);
  int32_t x[kUmItems];
  uint32_t vv[kUmItems];
  uint32_t keep = 0, first = 0;
  if (nitems) {
    uint32_t v = um_node(g, part[c].v, part[c + 1].v, pt);
    int64_t a0 = g.oo[v], b0 = g.io[v];
    uint32_t na = (uint32_t)(g.oo[v + 1] - a0), nb = (uint32_t)(g.io[v + 1] - b0);
    const uint32_t q = (uint32_t)(pt - (uint64_t)(a0 + b0));
    uint32_t i = um_path(g.on + a0, na, g.in + b0, nb, q), j = q - i;
    int32_t ca = i < na ? g.on[a0 + i] : INT32_MAX;    // next out-element
    int32_t cb = j < nb ? g.in[b0 + j] : INT32_MAX;    // next in-element
    int32_t la = i > 0 ? g.on[a0 + i - 1] : -1;        // last out-element taken
#pragma unroll
    for (uint32_t k = 0; k < kUmItems; ++k) {
      if (k < nitems) {
        while (i == na && j == nb) {  // this node is used up: on to the next with elements
          ++v;
          a0 = g.oo[v];
          b0 = g.io[v];
          na = (uint32_t)(g.oo[v + 1] - a0);
          nb = (uint32_t)(g.io[v + 1] - b0);
          i = j = 0;
          ca = na ? g.on[a0] : INT32_MAX;
          cb = nb ? g.in[b0] : INT32_MAX;
          la = -1;
        }
        first |= (uint32_t)(i == 0 && j == 0) << k;
        vv[k] = v;
        if (i < na && (j == nb || ca <= cb)) {
          x[k] = ca;
          la = ca;
          keep |= 1u << k;
          ++i;
          ca = i < na ? g.on[a0 + i] : INT32_MAX;
        } else {
          x[k] = cb;
          if (cb != la) keep |= 1u << k;
          ++j;
          cb = j < nb ? g.in[b0 + j] : INT32_MAX;
        }
      }
    }
  }
  uint32_t total;
  const uint32_t off = block_exclusive_sum<kUmThreads>((uint32_t)__popc(keep), s_sw, total);
  if constexpr (!WRITE) {
    if (threadIdx.x == 0) cnt[c] = total;
  } else {
    const int64_t b = base[c];
    uint32_t r = off;
#pragma unroll
    for (uint32_t k = 0; k < kUmItems; ++k) {
      if ((keep >> k) & 1u) {
        s_out[r] = x[k];
        if ((first >> k) & 1u) uoff[vv[k]] = b + r;
        ++r;
      }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < total; t += kUmThreads) unbr[b + t] = s_out[t];
    if (c == 0 && threadIdx.x == 0) uoff[g.V] = base[gridDim.x];
  }
}

uint32_t grid_of(uint64_t work, uint32_t per_block, uint32_t cap) {
  uint64_t g = (work + per_block - 1) / per_block;
  if (g == 0) g = 1;
  return (uint32_t)(g < cap ? g : cap);
}

}  // namespace

int build_undirected(const int64_t* out_off, const int32_t* out_nbr, const int64_t* in_off,
                     const int32_t* in_nbr, uint32_t V, uint64_t E, cudaStream_t s,
                     int64_t** und_off, int32_t** und_nbr, uint64_t* M) {
  *und_off = nullptr;
  *und_nbr = nullptr;
  *M = 0;
  const UmGraph g{out_off, out_nbr, in_off, in_nbr, V, 2 * E};
  const uint64_t nch64 = (g.W + kUmTile - 1) / kUmTile;
  if (V == 0 || nch64 == 0) {
    set_error("undirected merge: empty graph");
    return RINGO_EINVAL;
  }
  if (nch64 >= 0x7FFFFFFFull) {
    set_error("undirected merge: too many adjacency entries");
    return RINGO_ERANGE;
  }
  const uint32_t nch = (uint32_t)nch64;
  const uint32_t tiles = (nch + kScanTileNodes - 1) / kScanTileNodes;
  // scratch: splits[nch + 1], block counts[nch], block starts[nch + 1], tile sums[tiles + 1]
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bytes = al(sizeof(UmSplit) * ((size_t)nch + 1)) + al(4 * (size_t)nch) +
                       al(8 * ((size_t)nch + 1)) + al(8 * ((size_t)tiles + 1));
  char* buf = (char*)pool_alloc(bytes, s);
  int64_t* uoff = (int64_t*)pool_alloc(8 * ((size_t)V + 1), s);
  if (!buf || !uoff) {
    pool_free(buf, s);
    pool_free(uoff, s);
    set_error("undirected merge: device memory");
    return RINGO_ENOMEM;
  }
  char* p = buf;
  UmSplit* part = (UmSplit*)p;  p += al(sizeof(UmSplit) * ((size_t)nch + 1));
  uint32_t* cnt = (uint32_t*)p; p += al(4 * (size_t)nch);
  int64_t* base = (int64_t*)p;  p += al(8 * ((size_t)nch + 1));
  uint64_t* tsum = (uint64_t*)p;
  int rc = RINGO_OK;
  uint64_t total = 0;
  int32_t* unbr = nullptr;
  cudaError_t e;
  {
    ProfScope ps("undirected_count", s);
    k_um_partition<<<grid_of((uint64_t)nch + 1, 256, 152 * 32), 256, 0, s>>>(g, nch, part);
    k_um_merge<false><<<nch, kUmThreads, 0, s>>>(g, part, cnt, nullptr, nullptr, nullptr);
    k_tc_tile_sums<<<tiles, 256, 0, s>>>(cnt, nch, (uint64_t*)tsum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(tsum, tiles);
    k_tc_tile_scan<<<tiles, 256, 0, s>>>(cnt, nch, tsum, tiles, base);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, base + nch, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("undirected merge: ") + cudaGetErrorString(e));
    rc = RINGO_ECUDA;
  } else if (total > 0x7FFFFFFFFFull || !(unbr = (int32_t*)pool_alloc(4 * (size_t)total + 4, s))) {
    set_error("undirected merge: device memory for the lists");
    rc = RINGO_ENOMEM;
  } else {
    {
      ProfScope ps("undirected_write", s);
      k_um_merge<true><<<nch, kUmThreads, 0, s>>>(g, part, nullptr, base, uoff, unbr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("undirected merge: ") + cudaGetErrorString(e));
      rc = RINGO_ECUDA;
    }
  }
  pool_free(buf, s);
  if (rc != RINGO_OK) {
    pool_free(uoff, s);
    pool_free(unbr, s);
    return rc;
  }
  *und_off = uoff;
  *und_nbr = unbr;
  *M = total;
  return RINGO_OK;
}

int run_triangles(const int64_t* off, const int32_t* nbr, uint32_t V, uint64_t E, cudaStream_t s,
                  uint64_t* count) {
  *count = 0;
  if (V == 0 || E == 0) return RINGO_OK;
  const uint32_t tiles = (V + kScanTileNodes - 1) / kScanTileNodes;
  // scratch: deg[V], cnt[V], deg16[V], off+[V+1], tile sums[tiles+1], total,
  // the oriented lists in the undirected lists' slots (E entries), then
  // packed (at most E / 2 + V entries: every non-loop edge is kept at one end)
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t packed = E / 2 + V;
  const size_t bytes = al(4 * (size_t)V) * 2 + al(2 * (size_t)V) + al(8 * ((size_t)V + 1)) +
                       al(8 * ((size_t)tiles + 1)) + al(8) + al(4 * (size_t)E) + al(4 * packed);
  char* buf = (char*)pool_alloc(bytes, s);
  if (!buf) return RINGO_ENOMEM;
  char* p = buf;
  int32_t* deg = (int32_t*)p;       p += al(4 * (size_t)V);
  uint32_t* cnt = (uint32_t*)p;     p += al(4 * (size_t)V);
  uint16_t* deg16 = (uint16_t*)p;   p += al(2 * (size_t)V);
  int64_t* offp = (int64_t*)p;      p += al(8 * ((size_t)V + 1));
  uint64_t* tsum = (uint64_t*)p;    p += al(8 * ((size_t)tiles + 1));
  unsigned long long* total = (unsigned long long*)p;  p += al(8);
  int32_t* nbrs = (int32_t*)p;      p += al(4 * (size_t)E);
  int32_t* nbrp = (int32_t*)p;
  const uint32_t warp_grid = grid_of(V, 8, 152 * 64);
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(total, 0, 8, s);
  {
    ProfScope ps("triangles_orient", s);
    k_tc_degree<<<grid_of(V, 256, 8192), 256, 0, s>>>(off, V, deg, deg16);
    k_tc_fill<<<warp_grid, 256, 0, s>>>(off, nbr, deg, deg16, V, cnt, nbrs);
    k_tc_tile_sums<<<tiles, 256, 0, s>>>(cnt, V, tsum);
    k_scan_tile_sums<<<1, 1024, 0, s>>>(tsum, tiles);
    k_tc_tile_scan<<<tiles, 256, 0, s>>>(cnt, V, tsum, tiles, offp);
    k_tc_pack<<<warp_grid, 256, 0, s>>>(off, cnt, nbrs, offp, V, nbrp);
  }
  {
    ProfScope ps("triangles_count", s);
    k_tc_triangles<<<warp_grid, 256, 0, s>>>(offp, nbrp, V, total);
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, total, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("triangles: ") + cudaGetErrorString(e));
    rc = RINGO_ECUDA;
  }
  pool_free(buf, s);
  *count = (uint64_t)h;
  return rc;
}

}  // namespace ringo
