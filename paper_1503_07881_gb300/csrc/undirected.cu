// Undirected conversion and triangle counting (ringo_table_to_undirected_graph,
// ringo_graph_count_triangles): the paper's undirected workload (Section 4,
// Table "paralg": triangle counting on the undirected LiveJournal and
// Twitter2010 graphs).
//
// Undirected conversion: each row (s, d) is the edge {s, d}; the table with
// every row also reversed goes through the same directed conversion, so each
// node's list holds its neighbours once, sorted, and both CSR directions are
// the same symmetric lists (a self-loop appears once).
//
// Triangles: edges are oriented from the endpoint of smaller (degree, index)
// to the larger, which keeps every oriented list below sqrt(2E) entries; a
// triangle {a, b, c} with a < b < c in that order is counted exactly once, as
// c in both N+(a) and N+(b).  For each oriented edge (u, v) the shorter of
// N+(u), N+(v) is searched, element by element, in the longer (both sorted
// by node index).
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

__global__ void k_double_table(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                               uint32_t n, int32_t* __restrict__ s2, int32_t* __restrict__ d2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t a = src[i], b = dst[i];
    s2[i] = a;
    d2[i] = b;
    s2[(size_t)n + i] = b;
    d2[(size_t)n + i] = a;
  }
}

__global__ void k_tc_degree(const int64_t* __restrict__ off, uint32_t V, int32_t* __restrict__ deg) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
    deg[v] = (int32_t)(off[v + 1] - off[v]);
}

// u -> v when (deg u, u) < (deg v, v); self-loops dropped
__device__ __forceinline__ bool oriented(const int32_t* __restrict__ deg, int32_t du, uint32_t u,
                                         uint32_t v) {
  if (v == u) return false;
  const int32_t dv = __ldg(deg + v);
  return dv > du || (dv == du && v > u);
}

// cnt[u] = oriented out-degree; one warp per node
__global__ void __launch_bounds__(256)
    k_tc_count(const int64_t* __restrict__ off, const int32_t* __restrict__ nbr,
               const int32_t* __restrict__ deg, uint32_t V, uint32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < V;
       u += warps) {
    const int64_t a = off[u], b = off[u + 1];
    const int32_t du = deg[u];
    uint32_t c = 0;
    for (int64_t e = a + lane; e < b; e += 32) c += oriented(deg, du, (uint32_t)u, (uint32_t)nbr[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) cnt[u] = c;
  }
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

__global__ void k_tc_scan_tiles(uint64_t* __restrict__ tsum, uint32_t tiles) {
  // one thread: tile counts are few (V / 2048)
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t run = 0;
  for (uint32_t t = 0; t < tiles; ++t) {
    const uint64_t c = tsum[t];
    tsum[t] = run;
    run += c;
  }
  tsum[tiles] = run;
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

// oriented lists, in the order of the undirected lists (ascending index)
__global__ void __launch_bounds__(256)
    k_tc_fill(const int64_t* __restrict__ off, const int32_t* __restrict__ nbr,
              const int32_t* __restrict__ deg, uint32_t V, const int64_t* __restrict__ offp,
              int32_t* __restrict__ nbrp) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t u = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < V;
       u += warps) {
    const int64_t a = off[u], b = off[u + 1];
    const int32_t du = deg[u];
    int64_t w = offp[u];
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane;
      const uint32_t v = e < b ? (uint32_t)nbr[e] : 0u;
      const bool keep = e < b && oriented(deg, du, (uint32_t)u, v);
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) nbrp[w + __popc(m & lt)] = (int32_t)v;
      w += __popc(m);
    }
  }
}

// |A ∩ B| for sorted lists: each element of the shorter searched in the longer
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
  uint32_t c = 0, lo0 = 0;
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

uint32_t grid_of(uint64_t work, uint32_t per_block, uint32_t cap) {
  uint64_t g = (work + per_block - 1) / per_block;
  if (g == 0) g = 1;
  return (uint32_t)(g < cap ? g : cap);
}

}  // namespace

int launch_double_table(const int32_t* src, const int32_t* dst, uint32_t n, int32_t* s2, int32_t* d2,
                        cudaStream_t s) {
  if (n == 0) return RINGO_OK;
  k_double_table<<<grid_of(n, 256, 8192), 256, 0, s>>>(src, dst, n, s2, d2);
  RINGO_LAUNCH_CHECK("k_double_table");
  return RINGO_OK;
}

int run_triangles(const int64_t* off, const int32_t* nbr, uint32_t V, uint64_t E, cudaStream_t s,
                  uint64_t* count) {
  *count = 0;
  if (V == 0 || E == 0) return RINGO_OK;
  const uint32_t tiles = (V + kScanTileNodes - 1) / kScanTileNodes;
  // scratch: deg[V], cnt[V], off+[V+1], tile sums[tiles+1], total, nbr+[<= E]
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bytes = al(4 * (size_t)V) * 2 + al(8 * ((size_t)V + 1)) + al(8 * ((size_t)tiles + 1)) +
                       al(8) + al(4 * (size_t)E);
  char* buf = (char*)pool_alloc(bytes, s);
  if (!buf) return RINGO_ENOMEM;
  char* p = buf;
  int32_t* deg = (int32_t*)p;       p += al(4 * (size_t)V);
  uint32_t* cnt = (uint32_t*)p;     p += al(4 * (size_t)V);
  int64_t* offp = (int64_t*)p;      p += al(8 * ((size_t)V + 1));
  uint64_t* tsum = (uint64_t*)p;    p += al(8 * ((size_t)tiles + 1));
  unsigned long long* total = (unsigned long long*)p;  p += al(8);
  int32_t* nbrp = (int32_t*)p;
  const uint32_t warp_grid = grid_of(V, 8, 152 * 64);
  int rc = RINGO_OK;
  cudaError_t e = cudaMemsetAsync(total, 0, 8, s);
  {
    ProfScope ps("triangles_orient", s);
    k_tc_degree<<<grid_of(V, 256, 8192), 256, 0, s>>>(off, V, deg);
    k_tc_count<<<warp_grid, 256, 0, s>>>(off, nbr, deg, V, cnt);
    k_tc_tile_sums<<<tiles, 256, 0, s>>>(cnt, V, tsum);
    k_tc_scan_tiles<<<1, 32, 0, s>>>(tsum, tiles);
    k_tc_tile_scan<<<tiles, 256, 0, s>>>(cnt, V, tsum, tiles, offp);
    k_tc_fill<<<warp_grid, 256, 0, s>>>(off, nbr, deg, V, offp, nbrp);
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
