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

// histogram, out-sort dst passes, dst ranks, out-sort src passes, dedup.
// Afterwards E, Vs, Vd are final in every segment's control block.  Counter
// i belongs to the i-th launch of a run.
int enqueue_phase1(const Launch& L, cudaStream_t s) {
  static_assert(kSortTile == kScanTile, "sort and scan tiles are the same rows");
  uint32_t* c = L.counters;
  int k = 0;
  RINGO_ENQUEUE("histogram", launch_histogram(L, c + k++, s));
  RINGO_ENQUEUE("plan", launch_plan(L, 0, s));
  for (int p = 0; p < 4; ++p) RINGO_ENQUEUE("onesweep", launch_onesweep(L, 0, p, p, c + k++, s));
  RINGO_ENQUEUE("dst_rank", launch_dst_rank(L, c + k++, s));
  for (int p = 4; p < kOutPasses; ++p)
    RINGO_ENQUEUE("onesweep", launch_onesweep(L, 0, p, p, c + k++, s));
  RINGO_ENQUEUE("dedup", launch_dedup(L, c + k++, s));
  return RINGO_OK;
}

int enqueue_sort_only(const Launch& L, cudaStream_t s) {
  uint32_t* c = L.counters;
  int k = 0;
  RINGO_ENQUEUE("histogram", launch_histogram(L, c + k++, s));
  RINGO_ENQUEUE("plan", launch_plan(L, 0, s));
  for (int p = 0; p < 4; ++p) RINGO_ENQUEUE("onesweep", launch_onesweep(L, 0, p, p, c + k++, s));
  RINGO_ENQUEUE("dst_rank", launch_dst_rank(L, c + k++, s));
  for (int p = 4; p < kOutPasses; ++p)
    RINGO_ENQUEUE("onesweep", launch_onesweep(L, 0, p, p, c + k++, s));
  return RINGO_OK;
}

// merge splits, merge into the node list, block tables of the two rank
// maps, out-direction remap.  The out-CSR is complete afterwards.
int enqueue_phase2(const Launch& L, cudaStream_t s) {
  uint32_t* c = L.counters + 20;
  RINGO_ENQUEUE("phase2_maps", launch_phase2_maps(L, s));
  RINGO_ENQUEUE("merge_split", launch_merge_split(L, s));
  RINGO_ENQUEUE("merge", launch_merge(L, c + 0, s));
  RINGO_ENQUEUE("rank_blocks", launch_rank_blocks(L, c + 1, s));
  RINGO_ENQUEUE("sort_steps", launch_sort_steps(L, s));
  RINGO_ENQUEUE("remap", launch_remap(L, c + 2, s));
  return RINGO_OK;
}

// in-sort passes, destination-run starts with in_nbr written as node
// indices, then in_off from the destination-run starts.
int enqueue_phase3(const Launch& L, cudaStream_t s) {
  uint32_t* c = L.counters + 11;
  int k = 0;
  RINGO_ENQUEUE("plan", launch_plan(L, 1, s));
  for (int p = 0; p < kInPasses; ++p)
    RINGO_ENQUEUE("onesweep", launch_onesweep(L, 1, p, kOutPasses + p, c + k++, s));
  RINGO_ENQUEUE("dst_runs", launch_dst_runs(L, c + k++, s));
  RINGO_ENQUEUE("fill_in_off", launch_fill_in_off(L, c + k++, s));
  return RINGO_OK;
}

#undef RINGO_ENQUEUE

}  // namespace ringo
