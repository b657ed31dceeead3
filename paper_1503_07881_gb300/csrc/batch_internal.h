// Host-side pieces shared by batched conversion (batch.cu) and the request
// server (server.cu): the resident base table, predicate pairs, selection
// ranges and one captured wave of the multi-segment pipeline.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ringo.h"

// A base table clustered by (tag, ts) in library-owned device memory.
struct ringo_base {
  int device = 0;
  uint32_t n = 0;
  int32_t* src_c = nullptr;
  int32_t* dst_c = nullptr;
  int64_t* ts_c = nullptr;
  int32_t* tag_c = nullptr;
};

namespace ringo {

// Per-segment sizes read back after a wave.
struct SegResult {
  uint32_t V, E, Vs, Vd, err, out_passes, in_passes, pad;
};

// One (tag, window) pair of predicate `seg`: one contiguous range of
// clustered rows.
struct Pair {
  int32_t tag;
  int32_t seg;
  int64_t t0, t1;
};

// Ranges of all pairs: lo[] and cnt[] on the device and cnt[] on the host.
struct Ranges {
  char* block = nullptr;  // one pool allocation holding the device arrays
  uint32_t* lo = nullptr;
  uint32_t* cnt = nullptr;
  std::vector<uint32_t> h_cnt;
  std::vector<uint32_t> h_lo;  // filled when asked for
};

// One converted segment of a wave: its sizes and its arrays inside the
// wave's output block.
struct WaveSeg {
  SegResult res;
  uint32_t res_rows = 0;
  int32_t* node_ids = nullptr;
  int64_t* out_off = nullptr;
  int32_t* out_nbr = nullptr;
  int64_t* in_off = nullptr;
  int32_t* in_nbr = nullptr;
};

struct WaveResult {
  char* block = nullptr;  // output block; the caller frees it (also on error)
  std::vector<WaveSeg> seg;
  std::vector<int32_t> topk_ids;  // [nseg][2][k], k = the topk argument
  std::vector<int64_t> topk_degs;
};

int check_preds(const ringo_select* preds, int32_t npred);
// One pair per distinct tag of each predicate, in predicate order.
std::vector<Pair> make_pairs(const ringo_select* preds, int32_t npred);
// Binary searches of all pairs on s; blocks until h_cnt (and, if host_lo,
// h_lo) is on the host.  The caller frees r->block (also on error).
int select_ranges(const ringo_base* b, const std::vector<Pair>& pairs, cudaStream_t s, Ranges* r,
                  bool host_lo = false);
// Converts one wave: segment j holds pairs [first[j], first[j + 1]) of the
// range arrays (device d_lo/d_cnt, or, with d_lo == nullptr, host h_lo/h_cnt
// uploaded with the wave's other small tables).  topk > 0 adds the top-k of
// both directions of every graph.
int run_wave(const ringo_base* b, const uint32_t* d_lo, const uint32_t* d_cnt,
             const uint32_t* h_lo, const uint32_t* h_cnt, const std::vector<size_t>& first,
             uint32_t nseg, uint32_t topk, cudaStream_t s, WaveResult* out);
// Device bytes one segment of n rows takes in a wave (scratch and outputs),
// an upper bound used for admission by memory budget.
uint64_t wave_seg_bytes(uint32_t n, uint32_t topk);
// Output bytes of one segment of n rows (node arrays sized for V <= 2n).
uint64_t wave_seg_output_bytes(uint32_t n);

}  // namespace ringo
