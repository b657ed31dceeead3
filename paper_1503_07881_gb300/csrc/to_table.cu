// Graph -> table conversion (ringo_graph_to_edge_table, ringo_graph_to_node_table
// and their batch forms).
//
// Section 3.4, "Conversion of graphs to tables": a node table or an edge table
// is built by splitting the graph's nodes or edges among workers, each
// writing its part of a pre-allocated output.  Here the output columns are
// pre-allocated by the caller and every edge is one work item: a 2048-edge
// tile finds the nodes it spans with one binary search per end, marks where
// each of them starts inside the tile, and a max-scan gives every edge its
// row node; rows are written coalesced, in CSR order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ringo.h"
#include "device_util.cuh"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

namespace {

constexpr uint32_t kExpandTile = 2048;   // edges per tile
constexpr uint32_t kExpandWindow = 2048; // most nodes a tile resolves by the max-scan

// shared-memory slot of tile position p: one pad word after every 8, so the
// 8 consecutive positions of each thread fall in distinct banks across a warp
__device__ __forceinline__ uint32_t pad8(uint32_t p) { return p + (p >> 3); }

// largest r in [0, V) with off[r] <= e (off[0] = 0 <= e < off[V] = E)
__device__ __forceinline__ uint32_t owner(const int64_t* __restrict__ off, uint32_t V, uint64_t e) {
  uint32_t lo = 0, hi = V;  // off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((uint64_t)off[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Rows e of the edge table, in CSR order: key[e] = node_ids[row node],
// val[e] = node_ids[nbr[e]].  For the out-CSR that is (src, dst); for the
// in-CSR the caller swaps the columns.  Each node whose edges start inside
// the tile marks its start position with its index (the largest index wins,
// so a node with no edges yields to the next one starting at the same
// place), and an inclusive max-scan over the tile gives every edge its row
// node.
__global__ void __launch_bounds__(256)
    k_expand(const int32_t* __restrict__ node_ids, const int64_t* __restrict__ off,
             const int32_t* __restrict__ nbr, uint32_t V, uint64_t E, int32_t* __restrict__ key,
             int32_t* __restrict__ val) {
  constexpr uint32_t kPer = kExpandTile / 256;  // positions per thread in the scan
  __shared__ int32_t s_own[kExpandTile + kExpandTile / 8];
  __shared__ int32_t s_w[8];
  __shared__ uint32_t s_r0, s_r1;
  for (uint64_t e0 = (uint64_t)blockIdx.x * kExpandTile; e0 < E;
       e0 += (uint64_t)gridDim.x * kExpandTile) {
    const uint64_t e1 = min(e0 + kExpandTile, E);
    const uint32_t len = (uint32_t)(e1 - e0);
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t r = warp_owner(off, V, e0, threadIdx.x);
      if (threadIdx.x == 0) s_r0 = r;
    } else if (threadIdx.x < 64) {
      const uint32_t r = warp_owner(off, V, e1 - 1, threadIdx.x - 32);
      if (threadIdx.x == 32) s_r1 = r;
    }
    for (uint32_t t = threadIdx.x; t < kExpandTile + kExpandTile / 8; t += blockDim.x) s_own[t] = 0;
    __syncthreads();
    const uint32_t r0 = s_r0, r1 = s_r1;
    if (r1 - r0 + 1 <= kExpandWindow) {
      // nodes r0+1 .. r1 start inside the tile
      for (uint32_t r = r0 + 1 + threadIdx.x; r <= r1; r += blockDim.x) {
        const uint64_t p = (uint64_t)off[r] - e0;
        if (p < len) atomicMax(&s_own[pad8((uint32_t)p)], (int32_t)(r - r0));
      }
      __syncthreads();
      // inclusive max-scan of s_own (each thread 8 consecutive positions)
      const uint32_t base = threadIdx.x * kPer;
      int32_t run = 0;
#pragma unroll
      for (uint32_t q = 0; q < kPer; ++q) run = max(run, s_own[pad8(base + q)]);
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      int32_t incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl = max(incl, y);
      }
      if (lane == 31) s_w[warp] = incl;
      __syncthreads();
      int32_t carry = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
      if (lane == 0) carry = 0;
      for (int k = 0; k < warp; ++k) carry = max(carry, s_w[k]);
      __syncthreads();  // every thread has its carry before the positions are overwritten
      int32_t m = carry;
#pragma unroll
      for (uint32_t q = 0; q < kPer; ++q) {
        m = max(m, s_own[pad8(base + q)]);
        s_own[pad8(base + q)] = m;
      }
      __syncthreads();
      for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) {
        const uint64_t e = e0 + t;
        const uint32_t r = r0 + (uint32_t)s_own[pad8(t)];
        const int32_t mm = __ldcs(nbr + e);
        // streaming stores, so the written columns do not push node_ids out of L2
        __stcs(key + e, node_ids[r]);
        __stcs(val + e, (uint32_t)mm < V ? __ldg(node_ids + mm) : 0);
      }
    } else {  // the tile spans more nodes than the window: search per edge
      for (uint64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const uint32_t r = owner(off, V, e);
        const int32_t mm = __ldcs(nbr + e);
        key[e] = node_ids[r];
        val[e] = (uint32_t)mm < V ? __ldg(node_ids + mm) : 0;
      }
    }
  }
}

__global__ void k_node_table(const int32_t* __restrict__ node_ids, const int64_t* __restrict__ out_off,
                             const int64_t* __restrict__ in_off, uint32_t V, int32_t* __restrict__ ids,
                             int64_t* __restrict__ outdeg, int64_t* __restrict__ indeg) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < V; r += gridDim.x * blockDim.x) {
    ids[r] = node_ids[r];
    outdeg[r] = out_off[r + 1] - out_off[r];
    indeg[r] = in_off[r + 1] - in_off[r];
  }
}

}  // namespace

int launch_edge_table(const int32_t* node_ids, const int64_t* off, const int32_t* nbr, uint32_t V,
                      uint64_t E, int32_t* key, int32_t* val, cudaStream_t s) {
  if (E == 0) return RINGO_OK;
  uint64_t grid = (E + kExpandTile - 1) / kExpandTile;
  if (grid > 65535) grid = 65535;
  {
    ProfScope ps("edge_table", s);
    k_expand<<<(uint32_t)grid, 256, 0, s>>>(node_ids, off, nbr, V, E, key, val);
  }
  RINGO_LAUNCH_CHECK("k_expand");
  return RINGO_OK;
}

int launch_node_table(const int32_t* node_ids, const int64_t* out_off, const int64_t* in_off,
                      uint32_t V, int32_t* ids, int64_t* outdeg, int64_t* indeg, cudaStream_t s) {
  if (V == 0) return RINGO_OK;
  uint32_t grid = (V + 255) / 256;
  if (grid > 8192) grid = 8192;
  {
    ProfScope ps("node_table", s);
    k_node_table<<<grid, 256, 0, s>>>(node_ids, out_off, in_off, V, ids, outdeg, indeg);
  }
  RINGO_LAUNCH_CHECK("k_node_table");
  return RINGO_OK;
}

}  // namespace ringo
