// PageRank on a built graph (ringo_graph_pagerank): the paper's second
// workload (Section 4, Table "paralg": ten iterations on LiveJournal and
// Twitter2010).  Power iteration from the uniform vector, in fp64:
//
//   PR'(v) = (1 - d) / V + d * ( sum over in-neighbours u of PR(u) / outdeg(u)
//                                + (sum of PR over nodes without out-edges) / V ).
//
// Each node's sum over its in-edges is formed in a fixed order, so the
// result is the same on every run.  The in-edges are cut into 2048-edge
// tiles (whatever the node boundaries):
//   edges: each thread of a block gathers the contributions of 8
//          consecutive edges of the tile into registers (two 16-byte index
//          loads, 8 independent gathers), finds each edge's
//          node with a max-scan of node starts, and sums every node's run
//          with a segmented scan over the threads' 8-edge runs; a node that
//          lies inside the tile gets its sum written, a node cut by the tile
//          edges leaves a partial sum in the tile's two slots;
//   fix-up: one warp per node that ends in a tile it did not start in adds
//          its partial sums in tile order;
//   nodes: PR(v), the next contributions PR(v) * (1 / outdeg(v)), and
//          per-block sums of PR over nodes without out-edges, reduced in a
//          fixed order.
// The first and last node of every tile and the reciprocal out-degrees are
// found once per call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kPrTile = 2048;      // in-edges per tile of the edge pass
constexpr uint32_t kPrPer = kPrTile / 256;  // consecutive positions per thread
constexpr uint32_t kNodeGrid = 1024;   // blocks of the node pass (fixed: partial sums)

struct PrState {
  double dangling;  // sum of PR over nodes without out-edges, for this iteration
};

// shared-memory slot of tile position p: one pad slot after every 8, so each
// thread's 8 consecutive positions fall in distinct banks across a warp
__device__ __forceinline__ uint32_t pad8(uint32_t p) { return p + (p >> 3); }

// tnode[2t], tnode[2t + 1]: the nodes owning the first and the last in-edge
// of tile t.  One warp per tile.
__global__ void k_pr_tile_nodes(const int64_t* __restrict__ in_off, uint32_t V, uint64_t E,
                                uint32_t tiles, uint32_t* __restrict__ tnode) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles; t += warps) {
    const uint64_t e0 = (uint64_t)t * kPrTile;
    const uint64_t e1 = e0 + kPrTile < E ? e0 + kPrTile : E;
    const uint32_t a = warp_owner(in_off, V, e0, lane);
    const uint32_t b = warp_owner(in_off, V, e1 - 1, lane);
    if (lane == 0) {
      tnode[2 * t] = a;
      tnode[2 * t + 1] = b;
    }
  }
}

// The run of one node at the end of a range of tile positions: the range's
// first and last node (relative to the tile's first node) and the sum of the
// positions that belong to its last node.  Keys do not decrease along the
// tile, so the run of the concatenation AB is A's run plus B's when B holds
// one node only and that node is A's last, else B's run.
struct Run {
  int32_t kf, kl;
  double tail;
};

__device__ __forceinline__ Run run_cat(const Run& a, const Run& b) {
  Run r;
  r.kf = a.kf;
  r.kl = b.kl;
  r.tail = (b.kf == b.kl && a.kl == b.kf) ? a.tail + b.tail : b.tail;
  return r;
}

// One block per tile of kPrTile in-edges.  sum[v] for every node whose
// in-edges lie inside the tile; part[2t] = the tile's share of its first node
// when that node starts in an earlier tile, part[2t + 1] = the share of its
// last node when that node goes on past the tile.
__global__ void __launch_bounds__(256, 5)
    k_pr_edges(const int64_t* __restrict__ in_off, const int32_t* __restrict__ in_nbr, uint32_t V,
               uint64_t E, const uint32_t* __restrict__ tnode, const double* __restrict__ contrib,
               double* __restrict__ sum, double* __restrict__ part) {
  __shared__ int32_t s_own[kPrTile + kPrTile / 8];
  __shared__ int32_t s_kf[256];
  __shared__ int32_t s_wm[8];
  __shared__ Run s_wr[8];
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t t = blockIdx.x;
  const uint64_t e0 = (uint64_t)t * kPrTile;
  const uint32_t len = (uint32_t)(E - e0 < kPrTile ? E - e0 : kPrTile);
  const uint64_t e1 = e0 + len;
  const uint32_t r0 = tnode[2 * t], r1 = tnode[2 * t + 1];
  // where the first node starts and the last one ends: only these two can be
  // cut by the tile's edges
  const uint64_t a_first = (uint64_t)in_off[r0], b_last = (uint64_t)in_off[r1 + 1];
  // this thread's 8 consecutive in-neighbours (in flight while the marks are
  // placed); positions past the tile's end read as no neighbour
  const uint32_t base = tid * kPrPer;
  uint32_t u[kPrPer];
  const int32_t* nb = in_nbr + e0 + base;
  if (base + kPrPer <= len && (((uintptr_t)nb) & 15) == 0) {
    const int4 x = __ldcs(reinterpret_cast<const int4*>(nb));  // streamed: keep L2 for contrib
    const int4 y = __ldcs(reinterpret_cast<const int4*>(nb) + 1);
    u[0] = (uint32_t)x.x; u[1] = (uint32_t)x.y; u[2] = (uint32_t)x.z; u[3] = (uint32_t)x.w;
    u[4] = (uint32_t)y.x; u[5] = (uint32_t)y.y; u[6] = (uint32_t)y.z; u[7] = (uint32_t)y.w;
  } else {
#pragma unroll
    for (uint32_t j = 0; j < kPrPer; ++j) u[j] = base + j < len ? (uint32_t)nb[j] : 0xFFFFFFFFu;
  }
#pragma unroll
  for (uint32_t q = 0; q < kPrPer; ++q) s_own[pad8(q * 256 + tid)] = 0;
  __syncthreads();
  // nodes r0+1 .. r1 start inside the tile; where several start at the same
  // place (all but the last without in-edges) the last one wins
  for (uint32_t r = r0 + 1 + tid; r <= r1; r += 256) {
    const uint64_t p = (uint64_t)in_off[r] - e0;
    if (p < len) atomicMax(&s_own[pad8((uint32_t)p)], (int32_t)(r - r0));
  }
  // contributions of this thread's edges, kept in registers (0 past the end)
  double val[kPrPer];
#pragma unroll
  for (uint32_t j = 0; j < kPrPer; ++j) val[j] = u[j] < V ? __ldg(contrib + u[j]) : 0.0;
  __syncthreads();
  // inclusive max-scan of the marks: key[j] = node of position 8 tid + j
  int32_t key[kPrPer];
  int32_t mx = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPrPer; ++j) {
    key[j] = s_own[pad8(base + j)];
    mx = max(mx, key[j]);
  }
  int32_t incl = mx;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl = max(incl, y);
  }
  if (lane == 31) s_wm[warp] = incl;
  __syncthreads();
  int32_t m = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  if (lane == 0) m = 0;
  for (uint32_t k = 0; k < warp; ++k) m = max(m, s_wm[k]);
#pragma unroll
  for (uint32_t j = 0; j < kPrPer; ++j) {
    m = max(m, key[j]);
    key[j] = m;
  }
  // a node's share of the tile goes to its sum, or to one of the tile's two
  // slots when the tile's edges cut the node (only the first and the last
  // node can be cut: a node after the first starts inside the tile, a node
  // before the last ends inside it)
  auto emit = [&](int32_t k, double x) {
    const uint32_t v = r0 + (uint32_t)k;
    const bool cut_before = k == 0 && a_first < e0;
    const bool cut_after = v == r1 && b_last > e1;
    if (!cut_before && !cut_after) {
      sum[v] = x;
    } else {
      if (cut_before) part[2 * t] = x;
      if (cut_after) part[2 * t + 1] = x;
    }
  };
  // the runs of this thread's 8 edges, one add per edge: a run that both
  // starts and ends here is complete now; the first run may continue one of
  // earlier threads (`head`), the last may go on into later ones (`acc`)
  double head = 0.0, acc = val[0];
  bool closed = false;  // the first run ended inside this thread
#pragma unroll
  for (uint32_t j = 0; j + 1 < kPrPer; ++j) {
    if (key[j + 1] != key[j]) {
      if (closed) emit(key[j], acc);
      else head = acc;
      closed = true;
      acc = val[j + 1];
    } else {
      acc += val[j + 1];
    }
  }
  // segmented scan over threads of (first node, last node, sum of the last
  // node's positions)
  Run mine;
  mine.kf = key[0];
  mine.kl = key[kPrPer - 1];
  mine.tail = acc;
  Run inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Run y;
    y.kf = __shfl_up_sync(0xFFFFFFFFu, inc.kf, o);
    y.kl = __shfl_up_sync(0xFFFFFFFFu, inc.kl, o);
    y.tail = __shfl_up_sync(0xFFFFFFFFu, inc.tail, o);
    if ((int)lane >= o) inc = run_cat(y, inc);
  }
  s_kf[tid] = mine.kf;
  if (lane == 31) s_wr[warp] = inc;
  __syncthreads();
  // the run that ends just before this thread: earlier warps in order, then
  // the earlier lanes of this warp
  Run before;
  before.kf = -1;
  before.kl = -1;
  before.tail = 0.0;
  for (uint32_t k = 0; k < warp; ++k) before = k == 0 ? s_wr[0] : run_cat(before, s_wr[k]);
  Run prev;
  prev.kf = __shfl_up_sync(0xFFFFFFFFu, inc.kf, 1);
  prev.kl = __shfl_up_sync(0xFFFFFFFFu, inc.kl, 1);
  prev.tail = __shfl_up_sync(0xFFFFFFFFu, inc.tail, 1);
  if (lane > 0) before = warp == 0 ? prev : run_cat(before, prev);
  const int32_t next = tid + 1 < 256 ? s_kf[tid + 1] : 0x7FFFFFFF;  // node after this thread
  const bool carried = before.kl == key[0];  // the first run started in an earlier thread
  if (closed) {
    emit(key[0], carried ? before.tail + head : head);
    if (next != key[kPrPer - 1]) emit(key[kPrPer - 1], acc);
  } else if (next != key[0]) {  // one run over all 8 edges, ending here
    emit(key[0], carried ? before.tail + acc : acc);
  }
}

// Nodes cut by tile edges: one warp per tile m whose first node started in
// an earlier tile k and ends in m adds that node's shares, part[2k + 1] then
// part[2(k+1)] .. part[2m], in a fixed order.
__global__ void k_pr_fixup(const int64_t* __restrict__ in_off, uint64_t E,
                           const uint32_t* __restrict__ tnode, uint32_t tiles,
                           const double* __restrict__ part, double* __restrict__ sum) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t mt = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); mt < tiles; mt += warps) {
    const uint32_t v = tnode[2 * mt];
    const uint64_t e0 = (uint64_t)mt * kPrTile;
    const uint64_t e1 = e0 + kPrTile < E ? e0 + kPrTile : E;
    const uint64_t a = (uint64_t)in_off[v], b = (uint64_t)in_off[v + 1];
    if (!(a < e0 && b <= e1)) continue;
    const uint32_t k = (uint32_t)(a / kPrTile);
    double acc = 0.0;
    for (uint32_t u = k + 1 + lane; u <= mt; u += 32) acc += part[2 * u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) sum[v] = part[2 * k + 1] + acc;
  }
}

// inv_od[v] = 1 / outdeg(v), 0 for a node without out-edges (once per call:
// an fp64 division costs many times a multiplication on this part)
__global__ void k_pr_inv_outdeg(const int64_t* __restrict__ out_off, uint32_t V,
                                double* __restrict__ inv_od) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const int64_t od = out_off[v + 1] - out_off[v];
    inv_od[v] = od > 0 ? 1.0 / (double)od : 0.0;
  }
}

// New ranks; next contributions; block sums of dangling rank.
__global__ void __launch_bounds__(256)
    k_pr_nodes(const double* __restrict__ inv_od, uint32_t V, double damping, int first,
               const PrState* __restrict__ st, double* __restrict__ pr, double* __restrict__ sum,
               double* __restrict__ contrib, double* __restrict__ partial) {
  __shared__ double s_w[8];
  const double inv_v = 1.0 / (double)V;
  const double base = first ? 0.0 : (1.0 - damping) * inv_v + damping * st->dangling * inv_v;
  double dang = 0.0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const double p = first ? inv_v : base + damping * sum[v];
    pr[v] = p;
    const double inv = inv_od[v];
    contrib[v] = p * inv;
    if (inv == 0.0) dang += p;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dang += __shfl_xor_sync(0xFFFFFFFFu, dang, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = dang;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += s_w[k];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_pr_reduce(const double* __restrict__ partial, uint32_t n, PrState* st) {
  __shared__ double s[256];
  double t = 0.0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) t += partial[i];
  s[threadIdx.x] = t;
  __syncthreads();
  for (uint32_t k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->dangling = s[0];
}

}  // namespace

int run_pagerank(const int64_t* out_off, const int64_t* in_off, const int32_t* in_nbr, uint32_t V,
                 uint64_t E, double damping, int32_t iterations, double* rank, cudaStream_t s) {
  if (V == 0) return RINGO_OK;
  // scratch: contrib[V], sum[V] (zero: nodes without in-edges keep 0), node
  // partials[kNodeGrid], state, tile shares[2 * tiles], tile nodes[2 * tiles],
  // 1 / outdeg[V]
  const uint64_t tiles = (E + kPrTile - 1) / kPrTile;
  if (tiles > 0x7FFFFFFFull) return RINGO_ERANGE;
  const size_t bytes = 24 * (size_t)V + 8 * kNodeGrid + 256 + 16 * tiles + 8 * tiles + 64;
  char* buf = (char*)pool_alloc(bytes, s);
  if (!buf) return RINGO_ENOMEM;
  double* contrib = (double*)buf;
  double* sum = contrib + V;
  double* partial = sum + V;
  PrState* st = (PrState*)(partial + kNodeGrid);
  double* part = (double*)(st + 1);
  uint32_t* tnode = (uint32_t*)(part + 2 * tiles);
  double* inv_od = (double*)(tnode + 2 * tiles);  // 8-byte aligned: 8 * tiles bytes on
  const uint32_t node_blocks = (V + 255) / 256;
  const uint32_t node_grid = node_blocks < kNodeGrid ? node_blocks : kNodeGrid;
  const uint64_t tw = (tiles + 7) / 8;  // 8 warps per block, one tile each
  const uint32_t tile_grid = (uint32_t)(tw < 65535 ? (tw > 0 ? tw : 1) : 65535);
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, s);
  if (tiles) k_pr_tile_nodes<<<tile_grid, 256, 0, s>>>(in_off, V, E, (uint32_t)tiles, tnode);
  k_pr_inv_outdeg<<<node_grid, 256, 0, s>>>(out_off, V, inv_od);
  // iteration 0 sets the uniform vector and its contributions
  {
    ProfScope ps("pagerank_nodes", s);
    k_pr_nodes<<<node_grid, 256, 0, s>>>(inv_od, V, damping, 1, st, rank, sum, contrib, partial);
  }
  k_pr_reduce<<<1, 256, 0, s>>>(partial, node_grid, st);
  for (int32_t it = 0; it < iterations; ++it) {
    if (tiles) {
      ProfScope ps("pagerank_edges", s);
      k_pr_edges<<<(uint32_t)tiles, 256, 0, s>>>(in_off, in_nbr, V, E, tnode, contrib, sum, part);
      k_pr_fixup<<<tile_grid, 256, 0, s>>>(in_off, E, tnode, (uint32_t)tiles, part, sum);
    }
    {
      ProfScope ps("pagerank_nodes", s);
      k_pr_nodes<<<node_grid, 256, 0, s>>>(inv_od, V, damping, 0, st, rank, sum, contrib,
                                           partial);
    }
    k_pr_reduce<<<1, 256, 0, s>>>(partial, node_grid, st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("pagerank: ") + cudaGetErrorString(e));
    rc = RINGO_ECUDA;
  }
  pool_free(buf, s);
  return rc;
}

}  // namespace ringo
