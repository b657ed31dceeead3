// PageRank on a built graph (ringo_graph_pagerank): the paper's second
// workload (Section 4, Table "paralg": ten iterations on LiveJournal and
// Twitter2010).  Power iteration from the uniform vector, in fp64:
//
//   PR'(v) = (1 - d) / V + d * ( sum over in-neighbours u of PR(u) / outdeg(u)
//                                + (sum of PR over nodes without out-edges) / V ).
//
// One iteration is three launches:
//   edges: in-CSR tiles of 2048 edges; each thread sums the contributions of
//          its 8 consecutive in-edges per target node, the block adds its
//          threads' sums per node in shared memory, and one global add per
//          (tile, node) gives sum[v] (so a node with millions of in-edges gets
//          one add per tile, not per edge);
//   nodes: PR(v), the next contributions PR(v) / outdeg(v), sum[v] cleared,
//          and per-block sums of PR over nodes without out-edges;
//   reduce: those block sums in a fixed order (one block).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kPrTile = 2048;    // in-edges per tile
constexpr uint32_t kPrItems = 8;      // per thread
constexpr uint32_t kPrWindow = 2048;  // target nodes staged per tile
constexpr uint32_t kNodeGrid = 1024;  // blocks of the node pass (fixed: partial sums)

struct PrState {
  double dangling;  // sum of PR over nodes without out-edges, for this iteration
};

__device__ __forceinline__ uint32_t pr_owner(const int64_t* __restrict__ off, uint32_t V, uint64_t e) {
  uint32_t lo = 0, hi = V;  // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((uint64_t)off[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
    k_pr_edges(const int64_t* __restrict__ in_off, const int32_t* __restrict__ in_nbr, uint32_t V,
               uint64_t E, const double* __restrict__ contrib, double* __restrict__ sum) {
  __shared__ int64_t s_off[kPrWindow + 1];
  __shared__ double s_acc[kPrWindow];
  __shared__ uint32_t s_r0, s_r1;
  for (uint64_t e0 = (uint64_t)blockIdx.x * kPrTile; e0 < E; e0 += (uint64_t)gridDim.x * kPrTile) {
    const uint64_t e1 = min(e0 + kPrTile, E);
    __syncthreads();
    if (threadIdx.x == 0) s_r0 = pr_owner(in_off, V, e0);
    if (threadIdx.x == 32) s_r1 = pr_owner(in_off, V, e1 - 1);
    __syncthreads();
    const uint32_t r0 = s_r0, r1 = s_r1;
    const uint32_t w = r1 - r0 + 1;
    const bool staged = w <= kPrWindow;
    if (staged) {
      for (uint32_t t = threadIdx.x; t <= w; t += blockDim.x) s_off[t] = in_off[r0 + t];
      for (uint32_t t = threadIdx.x; t < w; t += blockDim.x) s_acc[t] = 0.0;
    }
    __syncthreads();
    const uint64_t a = e0 + (uint64_t)threadIdx.x * kPrItems;
    if (a < e1) {
      const uint64_t b = min(a + kPrItems, e1);
      // the target node of edge a
      uint32_t r;
      if (staged) {
        uint32_t lo = 0, hi = w;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((uint64_t)s_off[mid] <= a) lo = mid;
          else hi = mid;
        }
        r = r0 + lo;
      } else {
        r = pr_owner(in_off, V, a);
      }
      uint64_t next = staged ? (uint64_t)s_off[r - r0 + 1] : (uint64_t)in_off[r + 1];
      double acc = 0.0;
      for (uint64_t e = a; e < b; ++e) {
        while (e >= next) {  // the next target node (skipping nodes without in-edges)
          if (acc != 0.0) {
            if (staged) atomicAdd(&s_acc[r - r0], acc);
            else atomicAdd(&sum[r], acc);
          }
          acc = 0.0;
          ++r;
          next = staged ? (uint64_t)s_off[r - r0 + 1] : (uint64_t)in_off[r + 1];
        }
        const uint32_t u = (uint32_t)__ldcs(in_nbr + e);
        acc += u < V ? __ldg(contrib + u) : 0.0;
      }
      if (acc != 0.0) {
        if (staged) atomicAdd(&s_acc[r - r0], acc);
        else atomicAdd(&sum[r], acc);
      }
    }
    __syncthreads();
    if (staged)
      for (uint32_t t = threadIdx.x; t < w; t += blockDim.x)
        if (s_acc[t] != 0.0) atomicAdd(&sum[r0 + t], s_acc[t]);
  }
}

// New ranks; next contributions; sum cleared; block sums of dangling rank.
__global__ void __launch_bounds__(256)
    k_pr_nodes(const int64_t* __restrict__ out_off, uint32_t V, double damping, int first,
               const PrState* __restrict__ st, double* __restrict__ pr, double* __restrict__ sum,
               double* __restrict__ contrib, double* __restrict__ partial) {
  __shared__ double s_w[8];
  const double inv_v = 1.0 / (double)V;
  const double base = first ? 0.0 : (1.0 - damping) * inv_v + damping * st->dangling * inv_v;
  double dang = 0.0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const double p = first ? inv_v : base + damping * sum[v];
    pr[v] = p;
    sum[v] = 0.0;
    const int64_t od = out_off[v + 1] - out_off[v];
    contrib[v] = od > 0 ? p / (double)od : 0.0;
    if (od == 0) dang += p;
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
  // scratch: contrib[V], sum[V], partial[kNodeGrid], state
  const size_t bytes = 16 * (size_t)V + 8 * kNodeGrid + 256;
  char* buf = (char*)pool_alloc(bytes, s);
  if (!buf) return RINGO_ENOMEM;
  double* contrib = (double*)buf;
  double* sum = contrib + V;
  double* partial = sum + V;
  PrState* st = (PrState*)(partial + kNodeGrid);
  const uint32_t node_blocks = (V + 255) / 256;
  const uint32_t node_grid = node_blocks < kNodeGrid ? node_blocks : kNodeGrid;
  uint64_t eg = (E + kPrTile - 1) / kPrTile;
  const uint32_t edge_grid = (uint32_t)(eg == 0 ? 1 : (eg > 65535 ? 65535 : eg));
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, s);
  // iteration 0 sets the uniform vector and its contributions
  {
    ProfScope ps("pagerank_nodes", s);
    k_pr_nodes<<<node_grid, 256, 0, s>>>(out_off, V, damping, 1, st, rank, sum, contrib, partial);
  }
  k_pr_reduce<<<1, 256, 0, s>>>(partial, node_grid, st);
  for (int32_t it = 0; it < iterations; ++it) {
    if (E) {
      ProfScope ps("pagerank_edges", s);
      k_pr_edges<<<edge_grid, 256, 0, s>>>(in_off, in_nbr, V, E, contrib, sum);
    }
    {
      ProfScope ps("pagerank_nodes", s);
      k_pr_nodes<<<node_grid, 256, 0, s>>>(out_off, V, damping, 0, st, rank, sum, contrib,
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
