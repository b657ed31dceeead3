// Internal declarations shared by the CUDA translation units of libringo.
//
// Pipeline (the paper's sort-first conversion, Section 3.4, re-designed for
// one GB300): the two ID columns are packed into 64-bit keys (biased src in
// the high word, biased dst in the low word) and LSD radix sorted.  After the
// four passes over the dst digits the keys are in dst order; one streaming
// kernel then replaces each dst by its destination-run index (monotone, so
// the order is kept) and emits the distinct destination IDs.  The four src
// passes follow.  Adjacent duplicates are dropped while source runs are
// counted; the surviving edges, re-keyed as (dst-run, source-run), are stably
// sorted on the dst-run half; the two sorted ID lists are merged into the
// node list; destination-run starts give the in-offsets; finally both neighbour
// arrays go from run indices to node indices through monotone maps, almost
// always answered by a small block table that stays in L2.  Sizes that only
// the device knows (E, V, which radix passes are trivial) live in the device
// control block `Ctl`, so the launch sequence needs no host decisions
// between kernels except the one sync that sizes the node arrays.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ringo {

// ------------------------------------------------------------- constants --
constexpr int kRadixBits = 8;   // digit width of the out-sort passes
constexpr int kRadix = 1 << kRadixBits;
constexpr int kOutPasses = 8;   // 64-bit (src,dst) keys
constexpr int kInPasses = 4;    // dst half of the (dst, src-run) keys
// The in-sort may use 9-bit digits instead (SweepOpts::in_digit_bits): four
// positions cover 36 bits, and three already cover the dst-run index of any
// table with at most 2^27 distinct destinations.
constexpr int kMaxRadixBits = 9;
constexpr int kMaxRadix = 1 << kMaxRadixBits;
// Words per tile (and per chunk) row of the radix look-back, whatever the
// digit width of the pass: a pass of 2^b digits uses the first 2^b words.
constexpr int kStRow = kMaxRadix;
// Histogram words of one sort: 8 passes x 256 digits or 4 passes x 512.
constexpr int kHistWords = kOutPasses * kRadix;
static_assert(kInPasses * kMaxRadix <= kHistWords, "in-sort histograms fit");
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kChunkShift = 5;               // 32 tiles per look-back chunk
constexpr int kChunkTiles = 1 << kChunkShift;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096 keys
constexpr int kMergeItems = 8;
constexpr int kMergeTile = kScanThreads * kMergeItems;  // 2048 merged items

constexpr uint32_t kBias = 0x80000000u;  // int32 -> uint32 preserving order
constexpr int kMaxSteps = 256;           // see Ctl::step_j

// Ctl::err bits
constexpr uint32_t kErrLookback = 1u;   // a radix look-back wait gave up
constexpr uint32_t kErrScan = 2u;       // a scan look-back wait gave up
constexpr uint32_t kErrRemap = 4u;      // a run index outside its map (bug)

// A bounded wait: about a second at most before the kernel records an error.
// A control block may set a lower bound of its own (Ctl::spin_limit).
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
  uint32_t bits;              // digit width of the passes (8 or 9)
  uint64_t* result;           // buffer holding the sorted keys
  uint64_t* spare;            // the other ping-pong buffer
  // digit counts and exclusive starts: pass p, digit d at [(p << bits) + d]
  uint32_t hist[kHistWords];
  uint32_t base[kHistWords];
};

struct alignas(16) Ctl {
  // sizes (device-side truth)
  uint32_t n_rows;
  uint32_t E, Vs, Vd, V;
  uint32_t err;
  uint32_t spin_limit;        // bound of every device wait (0: kSpinLimit)
  // inputs
  const int32_t* src;
  const int32_t* dst;
  // workspace
  uint64_t* keysA;            // [n_rows + 1]
  uint64_t* keysB;            // [n_rows + 1]
  uint32_t* status[2];        // [status_rows][kStRow] each, alternating passes
  uint32_t status_rows;
  // chunk level of the radix look-back (kChunkTiles tiles per chunk), two
  // regions alternating with the passes like `status`:
  //   chunk_agg[c][d] = (tiles of chunk c that have added << 32) | digit-d
  //                     count they added; one 64-bit word, so a single load
  //                     tells whether the sum is complete
  //   chunk_inc[c][d] = kStInc | inclusive prefix of digit d through chunk c
  uint64_t* chunk_agg[2];     // [chunks][kStRow]
  uint32_t* chunk_inc[2];     // [chunks][kStRow]
  uint32_t chunk_rows;
  uint64_t* scan_status[3];   // [tiles] each: dedup, dst_rank, merge
  uint64_t* scan_chunk_agg[3];  // [chunks of those tiles] packed sums
  uint64_t* scan_chunk_inc[3];  // [chunks] inclusive prefix, flagged
  uint32_t* scan_chunk_cnt[3];  // [chunks] tiles that have added their sum
  int32_t* usrc;              // [n_rows + 1] distinct src IDs, ascending
  int32_t* usrc_start;        // [n_rows + 1] first out-edge of each source run (phase 3: n_fill records)
  int32_t* udst;              // [n_rows + 1] distinct dst IDs, ascending
  int32_t* udst_start;        // [n_rows + 1] first in-edge of each destination run
  PassDesc rank_step;         // dst -> dst-run index, between out-sort passes 3 and 4
  // run index -> node index (both monotone), with block tables:
  //   blk[k] = map[32k] | 0x80000000 when map[32k .. 32k+31] has no gap
  int32_t* src_rank;          // [Vs]
  int32_t* dst_rank;          // [Vd]
  uint32_t* src_blk;          // [ceil(Vs / 32)]
  uint32_t* dst_blk;          // [ceil(Vd / 32)]
  // The dst-run -> node map as steps: dst_rank[j] - j only grows, by one
  // for every node that is not a destination; where it changes, j and the
  // new difference.  Filled (unordered) by k_rank_blocks while there are at
  // most kMaxSteps, then sorted by k_sort_steps; n_steps counts them all, so
  // a larger count means the list is not used.
  uint32_t n_fill;            // long node ranges of in_off recorded in usrc_start (phase 3)
  uint32_t n_steps;
  uint32_t step_j[kMaxSteps];
  uint32_t step_off[kMaxSteps];
  // outputs
  int32_t* out_nbr;           // [n_rows] capacity
  int32_t* in_nbr;            // [n_rows] capacity
  int32_t* node_ids;          // [Vs + Vd] capacity
  int64_t* out_off;           // [Vs + Vd + 1] capacity
  int64_t* in_off;
  SortCtl out_sort;
  SortCtl in_sort;
  // used when this control block runs alone (a single table): its slot maps
  // and claim counters
  uint32_t solo_rows[2];
  uint32_t solo_merge[2];
  uint32_t solo_blocks[2];
  uint32_t solo_counters[32];
};

// Bytes of one region of the radix chunk look-back (aggregates, then
// prefixes), and its placement.
__host__ __device__ constexpr uint64_t radix_chunk_bytes(uint64_t chunks) {
  return 12ull * chunks * kStRow;
}
__host__ __device__ inline void place_radix_chunks(Ctl* c, int r, void* p, uint64_t chunks) {
  c->chunk_agg[r] = static_cast<uint64_t*>(p);
  c->chunk_inc[r] = reinterpret_cast<uint32_t*>(static_cast<char*>(p) + 8ull * chunks * kStRow);
}
// Bytes of one region of the radix tile look-back for `tiles` tiles.
__host__ __device__ constexpr uint64_t radix_status_bytes(uint64_t tiles) {
  return 4ull * tiles * kStRow;
}

// Merge-path splits of the merge tiles (phase 2).  They live in the in-CSR
// neighbour array, which only phase 3 writes: at most (2n + 2047) / 2048 + 1
// words, far below its n entries.
__host__ __device__ inline uint32_t* merge_splits(const Ctl* c) {
  return reinterpret_cast<uint32_t*>(c->in_nbr);
}

constexpr uint32_t kBlkDense = 0x80000000u;

constexpr int kBlkShift = 5;  // 32 map entries per block-table word

// ------------------------------------------------------- multi-segment map --
// Every pipeline kernel runs over a table of segments at once (one segment
// for a single table, thousands for a batch): segment s owns the global tile
// slots [start[s], start[s+1]) (look-back chunks count from the segment's own
// first tile), and blocks claim slots in increasing order from a per-launch
// counter, so a tile only ever waits on earlier tiles of its own segment, all
// claimed before it.
struct SegMap {
  const uint32_t* start;  // [nseg + 1], device
  uint32_t nseg;
};

// Choices of the radix pass that the tuner measures (tune.cu):
//   rank_method     0: peers by shared-memory lane masks (one atomic OR and
//                      one read per key), 1: peers by one warp ballot per
//                      digit bit (no shared memory, 32 ALU operations per
//                      key; no atomic conflicts when many keys share a digit),
//                   2: peers by one warp match instruction on the digit
//   prefetch_waves  how far ahead (in waves of resident blocks) each block
//                   asks L2 for a tile's input; 0: no prefetch
//   in_digit_bits   digit width of the in-sort passes, 8 or 9
struct SweepOpts {
  int32_t rank_method = 0;
  int32_t prefetch_waves = 1;
  int32_t in_digit_bits = 8;
};
// The radix pass resident blocks per SM of a variant (its launch bounds):
// 512-digit passes with lane masks need more shared memory than four fit.
__host__ __device__ constexpr uint32_t sweep_blocks_per_sm(int bits, int rank_method) {
  return (bits > 8 && rank_method == 0) ? 3u : 4u;
}

// The segment table and slot maps of one run, and its claim counters.
struct Launch {
  Ctl* ctls;              // [nseg] device control blocks
  SegMap rows;            // 4096-row tiles of each segment
  SegMap merge;           // 2048-item tiles of each segment's node merge
  SegMap blocks;          // 4096-word pieces of each segment's block tables
  uint32_t row_slots;     // rows.start[nseg]
  uint32_t nseg;
  uint32_t* counters;     // [kNumCounters] device, zero at the start of a run
  SweepOpts opts;         // radix pass variant
};
// merge.start and blocks.start are written on the device after phase 1
// (from Vs and Vd); their kernels are persistent and loop over the slots.
constexpr int kNumCounters = 32;

// A single table: one segment whose maps and counters live in its own block.
// `dctl` is the device address of the block, `h` its host copy (the row map
// is filled in `h`, which the caller uploads).
inline Launch solo_launch(Ctl* dctl, Ctl* h, uint32_t n_rows) {
  const uint32_t tiles = (n_rows + kSortTile - 1) / kSortTile;
  h->solo_rows[0] = 0;
  h->solo_rows[1] = tiles;
  Launch L;
  L.ctls = dctl;
  L.nseg = 1;
  L.rows = SegMap{dctl->solo_rows, 1};
  L.merge = SegMap{dctl->solo_merge, 1};
  L.blocks = SegMap{dctl->solo_blocks, 1};
  L.row_slots = tiles;
  L.counters = dctl->solo_counters;
  return L;
}

// The pass options for a run of `kind` (0: one table, 1: a batch wave) whose
// segments hold `rows` rows on average: the forced ones if set
// (ringo_sort_opts_force), else the tuned choice for this GPU and size
// class, else the defaults.  wave_rows (batches) likewise, 0 when none.
SweepOpts sort_opts_for(int kind, uint64_t rows);
int64_t tuned_wave_rows(uint64_t rows_per_pred);
// Keeps the forced pass options (ringo_sort_opts_force) of its construction
// and puts them back when it goes out of scope (tuners force candidates).
struct ForcedOptsGuard {
  ForcedOptsGuard();
  ~ForcedOptsGuard();
  bool was;
  SweepOpts saved;
};
// The pass variants the tuners measure, in this order: every rank method and
// prefetch distance with 8-bit in-sort digits, then every rank method with
// 9-bit in-sort digits at the best prefetch distance so far.  `best()` gives
// the best options measured so far; the walk stops once `ok()` is false.
template <class Measure, class Best, class Ok>
void for_each_candidate(Measure&& measure, Best&& best, Ok&& ok) {
  for (int r = 0; r <= 2; ++r) {
    for (int w = 0; w <= 2; ++w) {
      if (!ok()) return;
      SweepOpts o;
      o.rank_method = r;
      o.prefetch_waves = w;
      o.in_digit_bits = 8;
      measure(o);
    }
  }
  const int w = best().prefetch_waves;
  for (int r = 0; r <= 2; ++r) {
    if (!ok()) return;
    SweepOpts o;
    o.rank_method = r;
    o.prefetch_waves = w;
    o.in_digit_bits = 9;
    measure(o);
  }
}
// Records a tuned choice (in memory and, when a cache file is set, on disk).
void record_tuned(int kind, uint64_t rows, const SweepOpts& o, int64_t wave_rows, double ms,
                  int out_passes, int in_passes);

// --------------------------------------------------------- host launchers --
// Each enqueues one kernel on `s`; `counter` is the launch's claim counter.
void launch_histogram(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_plan(const Launch& L, int which, cudaStream_t s);
void launch_onesweep(const Launch& L, int which, int pass, int gpass, uint32_t* counter,
                     cudaStream_t s);
void launch_dst_rank(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_dedup(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_dst_runs(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_phase2_maps(const Launch& L, cudaStream_t s);
void launch_merge_split(const Launch& L, cudaStream_t s);
// graph -> table (to_table.cu); both return a ringo status
int launch_edge_table(const int32_t* node_ids, const int64_t* off, const int32_t* nbr, uint32_t V,
                      uint64_t E, int32_t* key, int32_t* val, cudaStream_t s);
int launch_node_table(const int32_t* node_ids, const int64_t* out_off, const int64_t* in_off,
                      uint32_t V, int32_t* ids, int64_t* outdeg, int64_t* indeg, cudaStream_t s);
// undirected conversion and triangles (undirected.cu); ringo statuses
// The undirected lists of a directed graph (its V nodes, E edges, both
// CSRs): each node's out- and in-list merged, a neighbour in both kept once.
// Allocates *und_off[V + 1] and *und_nbr[*M] from the pool (on stream s) and
// returns a ringo status; on failure nothing stays allocated.
int build_undirected(const int64_t* out_off, const int32_t* out_nbr, const int64_t* in_off,
                     const int32_t* in_nbr, uint32_t V, uint64_t E, cudaStream_t s,
                     int64_t** und_off, int32_t** und_nbr, uint64_t* M);
int run_triangles(const int64_t* off, const int32_t* nbr, uint32_t V, uint64_t E, cudaStream_t s,
                  uint64_t* count);
// PageRank (pagerank.cu); returns a ringo status
int run_pagerank(const int64_t* out_off, const int64_t* in_off, const int32_t* in_nbr, uint32_t V,
                 uint64_t E, double damping, int32_t iterations, double* rank, cudaStream_t s);
void launch_merge(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_rank_blocks(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_remap(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_fill_in_off(const Launch& L, uint32_t* counter, cudaStream_t s);
void launch_sort_steps(const Launch& L, cudaStream_t s);
void launch_degrees(const int32_t* node_ids, const int64_t* off, uint32_t V,
                    const int32_t* ids, uint32_t n, int64_t* deg, cudaStream_t s);
int launch_topk(const int32_t* node_ids, const int64_t* off, uint32_t V, uint32_t k,
                int32_t* d_ids, int64_t* d_degs, void* d_scratch, size_t scratch_bytes,
                cudaStream_t s);
size_t topk_scratch_bytes(uint32_t V, uint32_t k);

// The launch sequence, shared by every entry point (pipeline.cu).
//   phase 1: histogram .. out-sort, dedup; afterwards E, Vs, Vd are final
//   phase 2: node merge, block tables, out-direction remap; needs node
//            arrays and rank maps set in every control block (sized from Vs,
//            Vd or from upper bounds).  Afterwards V, node_ids, out_off and
//            out_nbr are final.
//   phase 3: in-sort, destination runs with the in-direction remap, in_off.
int enqueue_phase1(const Launch& L, cudaStream_t s);
int enqueue_phase2(const Launch& L, cudaStream_t s);
int enqueue_phase3(const Launch& L, cudaStream_t s);
// histogram, plan, the four dst passes, the rank step, the four src passes:
// the out-sort alone (its keys end in out_sort.result)
int enqueue_sort_only(const Launch& L, cudaStream_t s);
// one-time kernel attributes, set before any stream capture
void prepare_launches();

}  // namespace ringo
