// The kernel launch sequence of the table->graph conversion, shared by every
// entry point (ringo_table_to_graph, ringo_table_to_graph_noalloc).  The
// caller owns the memory and the control block; these functions only enqueue
// kernels on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ringo.h"
#include "host_util.h"
#include "ringo_internal.cuh"

namespace ringo {

#define RINGO_ENQUEUE(name, call)                                                 \
  do {                                                                            \
    {                                                                             \
      ProfScope _ps(name, s);                                                     \
      call;                                                                       \
    }                                                                             \
    cudaError_t _e = cudaGetLastError();                                          \
    if (_e != cudaSuccess) {                                                      \
      set_error(std::string("launch ") + name + ": " + cudaGetErrorString(_e));   \
      return RINGO_ECUDA;                                                         \
    }                                                                             \
  } while (0)

// histogram, out-sort dst passes, dst ranks, out-sort src passes, dedup,
// in-sort passes, destination-run starts.  Afterwards E, Vs, Vd are final.
int enqueue_phase1(Ctl* dctl, uint32_t n, cudaStream_t s) {
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
  static_assert(kSortTile == kScanTile, "sort and scan tiles are the same rows");
  RINGO_ENQUEUE("histogram", launch_histogram(dctl, n, s));
  RINGO_ENQUEUE("plan", launch_plan(dctl, 0, s));
  for (int p = 0; p < 4; ++p) RINGO_ENQUEUE("onesweep", launch_onesweep(dctl, 0, p, p, tiles, s));
  RINGO_ENQUEUE("dst_rank", launch_dst_rank(dctl, tiles, s));
  for (int p = 4; p < kOutPasses; ++p)
    RINGO_ENQUEUE("onesweep", launch_onesweep(dctl, 0, p, p, tiles, s));
  RINGO_ENQUEUE("dedup", launch_dedup(dctl, tiles, s));
  RINGO_ENQUEUE("plan", launch_plan(dctl, 1, s));
  for (int p = 0; p < kInPasses; ++p)
    RINGO_ENQUEUE("onesweep", launch_onesweep(dctl, 1, p, kOutPasses + p, tiles, s));
  RINGO_ENQUEUE("dst_runs", launch_dst_runs(dctl, n, s));
  return RINGO_OK;
}

// merge into the node list, block tables of the two rank maps, remap.
int enqueue_phase2(Ctl* dctl, uint32_t Vs, uint32_t Vd, uint32_t E, cudaStream_t s) {
  const uint64_t M = (uint64_t)Vs + Vd;
  const uint32_t mgrid = (uint32_t)((M + kMergeTile - 1) / kMergeTile);
  RINGO_ENQUEUE("merge", launch_merge(dctl, mgrid, s));
  RINGO_ENQUEUE("rank_blocks", launch_rank_blocks(dctl, Vs, Vd, s));
  RINGO_ENQUEUE("remap", launch_remap(dctl, E, s));
  return RINGO_OK;
}

#undef RINGO_ENQUEUE

}  // namespace ringo
