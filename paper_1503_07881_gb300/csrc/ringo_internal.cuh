// Internal declarations shared by the CUDA translation units of libringo.
//
// Pipeline (the paper's sort-first conversion, Section 3.4, re-designed for
// one GB300): the two ID columns are packed into 64-bit keys (biased src in
// the high word, biased dst in the low word) and LSD radix sorted; adjacent
// duplicates are dropped while source runs are counted; the surviving edges,
// re-keyed as (dst, source-run index), are stably sorted on the dst bits; the
// destination runs are counted; the sorted source and destination ID lists are
// merged into the node list; finally neighbour IDs are turned into node
// indices.  Every step is a kernel below; sizes that only the device knows
// (E, V, which radix passes are trivial) live in the device control block
// `Ctl`, so the launch sequence needs no host decisions between kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ringo {

// ------------------------------------------------------------- constants --
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kOutPasses = 8;   // 64-bit (src,dst) keys
constexpr int kInPasses = 4;    // dst half of the (dst, src-run) keys
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kSortWarps = kSortThreads / 32;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096 keys
constexpr int kMergeItems = 8;
constexpr int kMergeTile = kScanThreads * kMergeItems;  // 2048 merged items

constexpr uint32_t kBias = 0x80000000u;  // int32 -> uint32 preserving order

// Ctl::err bits
constexpr uint32_t kErrLookback = 1u;   // a radix look-back wait gave up
constexpr uint32_t kErrScan = 2u;       // a scan look-back wait gave up
constexpr uint32_t kErrRemap = 4u;      // an ID missing from node_ids (bug)

constexpr uint32_t kRankDirectory = 0;
constexpr uint32_t kRankBitmap = 1;
constexpr uint32_t kSectorIds = 224;  // ID bits per 32-byte rank sector

// A bounded wait: about a second at most before the kernel records an error.
constexpr uint32_t kSpinLimit = 1u << 21;

// radix look-back status word (one per tile and digit), 32 bits:
//   0                 not yet published
//   1 + count         tile aggregate only (count <= kSortTile)
//   0x80000000 | sum  inclusive prefix (sum < 2^31)
constexpr uint32_t kStInc = 0x80000000u;

// scan look-back status word (one per tile), 64 bits:
//   bits 63..62 flag (1 aggregate, 2 inclusive), bits 61..31 count A,
//   bits 30..0 count B.  Packed values add without carries between fields
//   because every total is below 2^31.
constexpr uint64_t kScanAgg = 1ull << 62;
constexpr uint64_t kScanInc = 2ull << 62;
constexpr uint64_t kScanValMask = (1ull << 62) - 1;
__host__ __device__ constexpr uint64_t pack2(uint32_t a, uint32_t b) {
  return ((uint64_t)a << 31) | (uint64_t)b;
}
__host__ __device__ constexpr uint32_t unpackA(uint64_t v) {
  return (uint32_t)((v >> 31) & 0x7FFFFFFFu);
}
__host__ __device__ constexpr uint32_t unpackB(uint64_t v) {
  return (uint32_t)(v & 0x7FFFFFFFu);
}

// ---------------------------------------------------------- control block --
struct PassDesc {
  const uint64_t* in;  // NULL: pack keys from the src/dst columns
  uint64_t* out;
  uint32_t shift;
  uint32_t active;     // 0: every key has the same digit; the pass is skipped
};

struct SortCtl {
  PassDesc pass[kOutPasses];
  uint32_t n;                 // keys to sort
  uint32_t active_passes;
  uint64_t* result;           // buffer holding the sorted keys
  uint64_t* spare;            // the other ping-pong buffer
  uint32_t hist[kOutPasses][kRadix];
  uint32_t base[kOutPasses][kRadix];
  uint32_t tile_counter[kOutPasses];
};

struct Ctl {
  // sizes (device-side truth)
  uint32_t n_rows;
  uint32_t E, Vs, Vd, V;
  uint32_t err;
  uint32_t scan_counter[4];   // dynamic tile counters: dedup, dst runs, merge
  // inputs
  const int32_t* src;
  const int32_t* dst;
  // workspace
  uint64_t* keysA;            // [n_rows + 1]
  uint64_t* keysB;            // [n_rows + 1]
  uint32_t* status[2];        // [status_rows][kRadix] each, alternating passes
  uint32_t status_rows;
  uint64_t* scan_status[3];   // [tiles] each: dedup, dst runs, merge
  int32_t* usrc;              // [n_rows + 1] distinct src IDs, ascending
  int32_t* usrc_start;        // [n_rows + 1] first edge of each src run
  int32_t* udst;              // distinct dst IDs (placed in the spare buffer)
  int32_t* udst_start;        // first in-edge of each dst run
  int32_t* src_rank;          // [Vs] node index of usrc[i]
  uint32_t id_lo, id_hi;      // smallest / largest biased ID in either column
  // ID -> node index, one of two structures (rank_mode):
  //  kRankDirectory: dir[k] = first node at or above bucket k of the ID range
  //  kRankBitmap:    32-byte sectors of {node count below the sector, 224 ID
  //                  bits}; one sector read answers a lookup
  uint32_t rank_mode;
  int32_t* dir;               // [dir_buckets + 1]
  uint32_t dir_buckets;       // power of two
  uint32_t* bitmap;           // [bitmap_sectors * 8]
  uint32_t bitmap_sectors;
  // outputs
  int32_t* out_nbr;           // [n_rows] capacity
  int32_t* in_nbr;            // [n_rows] capacity
  int32_t* node_ids;          // [Vs + Vd] capacity
  int64_t* out_off;           // [Vs + Vd + 1] capacity
  int64_t* in_off;
  SortCtl out_sort;
  SortCtl in_sort;
};

// --------------------------------------------------------- host launchers --
// Each enqueues one kernel on `s`; `ctl` is the device copy of the block.
void launch_histogram(Ctl* ctl, uint32_t n_rows, cudaStream_t s);
void launch_plan(Ctl* ctl, int which, cudaStream_t s);
void launch_onesweep(Ctl* ctl, int which, int pass, int gpass, uint32_t grid, cudaStream_t s);
void launch_dedup(Ctl* ctl, uint32_t grid, cudaStream_t s);
void launch_dst_runs(Ctl* ctl, uint32_t grid, cudaStream_t s);
void launch_merge(Ctl* ctl, uint32_t grid, cudaStream_t s);
void launch_directory(Ctl* ctl, uint32_t V, cudaStream_t s);
void launch_rank_bitmap(Ctl* ctl, uint32_t V, cudaStream_t s);
void launch_remap(Ctl* ctl, uint32_t E, uint32_t mode, cudaStream_t s);
void launch_degrees(const int32_t* node_ids, const int64_t* off, uint32_t V,
                    const int32_t* ids, uint32_t n, int64_t* deg, cudaStream_t s);
int launch_topk(const int32_t* node_ids, const int64_t* off, uint32_t V, uint32_t k,
                int32_t* d_ids, int64_t* d_degs, void* d_scratch, size_t scratch_bytes,
                cudaStream_t s);
size_t topk_scratch_bytes(uint32_t V, uint32_t k);

}  // namespace ringo
