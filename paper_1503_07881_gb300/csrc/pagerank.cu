// PageRank on a built graph (ringo_graph_pagerank): the paper's second
// workload (Section 4, Table "paralg": ten iterations on LiveJournal and
// Twitter2010).  Power iteration from the uniform vector, in fp64:
//
//   PR'(v) = (1 - d) / V + d * ( sum over in-neighbours u of PR(u) / outdeg(u)
//                                + (sum of PR over nodes without out-edges) / V ).
//
// Each node's sum over its in-edges is formed in a fixed order, so the
// result is the same on every run:
//   light nodes (in-degree up to kBig): one warp per node, lanes striding over
//          its in-edges (coalesced index loads, independent gathers), a
//          fixed-order warp reduction, one plain store;
//   heavy nodes: split into kBig-edge chunks, one block per chunk with a
//          fixed-order block reduction, then the chunks of each node added in
//          order;
//   nodes: PR(v), the next contributions PR(v) / outdeg(v), and per-block
//          sums of PR over nodes without out-edges, reduced in a fixed order.
// The heavy-node list and its chunk offsets are built once per call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kBig = 8192;        // in-edges above which a node is split into chunks
constexpr uint32_t kNodeGrid = 1024;   // blocks of the node pass (fixed: partial sums)

struct PrState {
  double dangling;  // sum of PR over nodes without out-edges, for this iteration
};

// Light nodes: one warp per node (grid-stride over warps).  sum[v] is
// written for every node of in-degree at most kBig, 0 when it has none.
__global__ void __launch_bounds__(256)
    k_pr_light(const int64_t* __restrict__ in_off, const int32_t* __restrict__ in_nbr, uint32_t V,
               const double* __restrict__ contrib, double* __restrict__ sum) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t v = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < V;
       v += warps) {
    const int64_t a = in_off[v], b = in_off[v + 1];
    if (b - a > (int64_t)kBig) continue;  // heavy: summed by chunks
    double acc = 0.0;
    int64_t e = a + lane;
    for (; e + 96 < b; e += 128) {  // four independent gathers in flight per lane
      const uint32_t u0 = (uint32_t)__ldcs(in_nbr + e), u1 = (uint32_t)__ldcs(in_nbr + e + 32);
      const uint32_t u2 = (uint32_t)__ldcs(in_nbr + e + 64), u3 = (uint32_t)__ldcs(in_nbr + e + 96);
      const double c0 = u0 < V ? __ldg(contrib + u0) : 0.0, c1 = u1 < V ? __ldg(contrib + u1) : 0.0;
      const double c2 = u2 < V ? __ldg(contrib + u2) : 0.0, c3 = u3 < V ? __ldg(contrib + u3) : 0.0;
      acc += (c0 + c1) + (c2 + c3);
    }
    for (; e < b; e += 32) {
      const uint32_t u = (uint32_t)__ldcs(in_nbr + e);
      acc += u < V ? __ldg(contrib + u) : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) sum[v] = acc;
  }
}

// The heavy nodes (in-degree above kBig), in any order, and their count.
__global__ void k_pr_heavy_list(const int64_t* __restrict__ in_off, uint32_t V, uint32_t* heavy,
                                uint32_t* nheavy) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
    if (in_off[v + 1] - in_off[v] > (int64_t)kBig) heavy[atomicAdd(nheavy, 1u)] = v;
}

// chunk_start[i] = chunks of heavy nodes before heavy[i]; chunk_start[n] = all.  One block.
__global__ void k_pr_chunk_starts(const int64_t* __restrict__ in_off, const uint32_t* __restrict__ heavy,
                                  const uint32_t* __restrict__ nheavy, uint32_t* chunk_start) {
  __shared__ uint32_t s_sw[33];
  __shared__ uint32_t carry;
  const uint32_t n = *nheavy;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < n; b0 += blockDim.x) {
    const uint32_t i = b0 + threadIdx.x;
    uint32_t c = 0;
    if (i < n) {
      const uint32_t v = heavy[i];
      c = (uint32_t)((in_off[v + 1] - in_off[v] + kBig - 1) / kBig);
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_sum<1024>(c, s_sw, tot);
    if (i < n) chunk_start[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) chunk_start[n] = carry;
}

// One block per chunk of kBig in-edges of a heavy node: a fixed-order sum.
__global__ void __launch_bounds__(256)
    k_pr_heavy_chunks(const int64_t* __restrict__ in_off, const int32_t* __restrict__ in_nbr,
                      uint32_t V, const double* __restrict__ contrib,
                      const uint32_t* __restrict__ heavy, const uint32_t* __restrict__ nheavy,
                      const uint32_t* __restrict__ chunk_start, double* __restrict__ partial) {
  __shared__ double s[256];
  __shared__ uint32_t s_i;
  const uint32_t n = *nheavy;
  const uint32_t total = chunk_start[n];
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {  // heavy node owning chunk g: last i with chunk_start[i] <= g
      uint32_t lo = 0, hi = n;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (chunk_start[mid] <= g) lo = mid;
        else hi = mid;
      }
      s_i = lo;
    }
    __syncthreads();
    const uint32_t i = s_i, v = heavy[i];
    const int64_t a = in_off[v] + (int64_t)(g - chunk_start[i]) * kBig;
    const int64_t b = min(a + (int64_t)kBig, in_off[v + 1]);
    double acc = 0.0;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
      const uint32_t u = (uint32_t)__ldcs(in_nbr + e);
      acc += u < V ? __ldg(contrib + u) : 0.0;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (uint32_t k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[g] = s[0];
  }
}

// sum[heavy node] = its chunks' sums, in chunk order.
__global__ void k_pr_heavy_sum(const uint32_t* __restrict__ heavy, const uint32_t* __restrict__ nheavy,
                               const uint32_t* __restrict__ chunk_start,
                               const double* __restrict__ partial, double* __restrict__ sum) {
  const uint32_t n = *nheavy;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (uint32_t g = chunk_start[i]; g < chunk_start[i + 1]; ++g) t += partial[g];
    sum[heavy[i]] = t;
  }
}

// New ranks; next contributions; block sums of dangling rank.
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
  // scratch: contrib[V], sum[V], node partials[kNodeGrid], state, heavy list
  // [V/kBig + 1], chunk starts [V/kBig + 2], chunk partials [E/kBig + V/kBig + 1]
  const uint64_t max_heavy = E / kBig + 1;
  const uint64_t max_chunks = E / kBig + max_heavy + 1;
  const size_t bytes = 16 * (size_t)V + 8 * kNodeGrid + 256 + 4 * (max_heavy + 1) +
                       4 * (max_heavy + 2) + 8 * max_chunks + 64;
  char* buf = (char*)pool_alloc(bytes, s);
  if (!buf) return RINGO_ENOMEM;
  double* contrib = (double*)buf;
  double* sum = contrib + V;
  double* partial = sum + V;
  double* cpartial = partial + kNodeGrid;
  PrState* st = (PrState*)(cpartial + max_chunks);
  uint32_t* nheavy = (uint32_t*)(st + 1);
  uint32_t* heavy = nheavy + 4;
  uint32_t* chunk_start = heavy + max_heavy + 1;
  const uint32_t node_blocks = (V + 255) / 256;
  const uint32_t node_grid = node_blocks < kNodeGrid ? node_blocks : kNodeGrid;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t lw = ((uint64_t)V + 7) / 8;  // 8 warps per block, one node each
  const uint32_t light_grid = (uint32_t)(lw < (uint64_t)sms * 64 ? lw : (uint64_t)sms * 64);
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, s);
  k_pr_heavy_list<<<node_grid, 256, 0, s>>>(in_off, V, heavy, nheavy);
  k_pr_chunk_starts<<<1, 1024, 0, s>>>(in_off, heavy, nheavy, chunk_start);
  // iteration 0 sets the uniform vector and its contributions
  {
    ProfScope ps("pagerank_nodes", s);
    k_pr_nodes<<<node_grid, 256, 0, s>>>(out_off, V, damping, 1, st, rank, sum, contrib, partial);
  }
  k_pr_reduce<<<1, 256, 0, s>>>(partial, node_grid, st);
  for (int32_t it = 0; it < iterations; ++it) {
    {
      ProfScope ps("pagerank_edges", s);
      k_pr_light<<<light_grid, 256, 0, s>>>(in_off, in_nbr, V, contrib, sum);
      if (E > kBig) {
        k_pr_heavy_chunks<<<(uint32_t)sms * 4, 256, 0, s>>>(in_off, in_nbr, V, contrib, heavy, nheavy,
                                                            chunk_start, cpartial);
        k_pr_heavy_sum<<<64, 256, 0, s>>>(heavy, nheavy, chunk_start, cpartial, sum);
      }
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
