// ringo_table_to_graph_noalloc: the table->graph conversion for callers that
// cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc (or any allocator) at the
// point where they convert a table: code running under a fixed device-memory
// budget that was reserved up front, a serving loop that must never block in
// the allocator or fragment the pool, or a host thread that already holds
// all the device memory it is allowed.  This entry point runs the same
// kernels as ringo_table_to_graph, but every scratch buffer lives in one
// file-scope __device__ array of fixed size, and the caller passes the output
// buffers.  It allocates no device or pinned host memory.
//
// The scratch array (g_noalloc_scratch, about 41 MB) exists once on every GPU
// where this library's device code is loaded and stays there until the
// process exits.  With CUDA's lazy module loading (the default) that happens
// on the first call on each device: its address is looked up then
// (cudaGetSymbolAddress, with that device current), which makes the driver
// load the module and place the array, so that first call does take device
// memory and can fail with RINGO_ENOMEM when none is left.  Callers make it
// at set-up time, while memory is still free.  Every call blocks (it
// synchronises the stream twice and reads sizes back in between), so no call
// can be made inside a stream capture.  All calls share the array: two calls
// whose work overlaps on the GPU (different streams or threads) race and
// corrupt each other's results; callers must serialise them.  The array
// keeps whatever the last call left in it, so each call clears the parts
// that must start at zero.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/ringo.h"
#include "host_util.h"
#include "ringo_internal.cuh"

using namespace ringo;

namespace {

constexpr uint32_t kMaxRows = RINGO_NOALLOC_MAX_ROWS;
constexpr size_t kA = 256;
constexpr size_t up(size_t x) { return (x + kA - 1) & ~(kA - 1); }
constexpr size_t up4(size_t x) { return (x + 3) & ~(size_t)3; }
constexpr size_t kTiles = (kMaxRows + kSortTile - 1) / kSortTile;
constexpr size_t kMergeTiles = (2 * (size_t)kMaxRows + kMergeTile - 1) / kMergeTile + 1;
// rank maps of at most kMaxRows sources and destinations, and their tables
constexpr size_t kRankWords = 2 * up4(kMaxRows) + 2 * up4((kMaxRows + 31) / 32);

constexpr size_t kOffCtl = 0;
constexpr size_t kOffKeysA = up(kOffCtl + sizeof(Ctl));
constexpr size_t kOffKeysB = up(kOffKeysA + 8 * ((size_t)kMaxRows + 1));
constexpr size_t kOffSt0 = up(kOffKeysB + 8 * ((size_t)kMaxRows + 1));
constexpr size_t kOffSt1 = up(kOffSt0 + radix_status_bytes(kTiles));
constexpr size_t kChunks = (kTiles + kChunkTiles - 1) / kChunkTiles;
constexpr size_t kChunkBytes = up(radix_chunk_bytes(kChunks));
constexpr size_t kOffCh0 = up(kOffSt1 + radix_status_bytes(kTiles));
constexpr size_t kOffCh1 = up(kOffCh0 + kChunkBytes);
constexpr size_t kOffSc0 = up(kOffCh1 + kChunkBytes);
constexpr size_t chunks_for(size_t tiles) { return (tiles + kChunkTiles - 1) / kChunkTiles; }
constexpr size_t scan_bytes(size_t tiles) {
  return up(8 * tiles) + up(8 * chunks_for(tiles)) * 2 + up(4 * chunks_for(tiles));
}
constexpr size_t kOffSc1 = up(kOffSc0 + scan_bytes(kTiles));
constexpr size_t kOffSc2 = up(kOffSc1 + scan_bytes(kTiles));
constexpr size_t kOffUsrc = up(kOffSc2 + scan_bytes(kMergeTiles));

void place_scan(Ctl* h, int i, unsigned char* p, size_t tiles) {
  const size_t c = chunks_for(tiles);
  h->scan_status[i] = (uint64_t*)p;
  p += up(8 * tiles);
  h->scan_chunk_agg[i] = (uint64_t*)p;
  p += up(8 * c);
  h->scan_chunk_inc[i] = (uint64_t*)p;
  p += up(8 * c);
  h->scan_chunk_cnt[i] = (uint32_t*)p;
}
constexpr size_t kOffUsrcStart = up(kOffUsrc + 4 * ((size_t)kMaxRows + 1));
constexpr size_t kOffUdst = up(kOffUsrcStart + 4 * ((size_t)kMaxRows + 1));
constexpr size_t kOffUdstStart = up(kOffUdst + 4 * ((size_t)kMaxRows + 1));
constexpr size_t kOffRanks = up(kOffUdstStart + 4 * ((size_t)kMaxRows + 1));
constexpr size_t kScratchBytes = up(kOffRanks + 4 * kRankWords);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("ringo_table_to_graph_noalloc: no usable current device");
    return RINGO_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                cudaGetErrorString(e));
      // placing the array (first call on this device) needs device memory
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RINGO_ENOMEM;
      }
      return RINGO_ECUDA;
    }
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_addr[dev];
  return RINGO_OK;
}

}  // namespace

extern "C" int ringo_table_to_graph_noalloc(const int32_t* src, const int32_t* dst,
                                            int64_t nrows, void* stream, int32_t* node_ids,
                                            int64_t* out_off, int32_t* out_nbr,
                                            int64_t* in_off, int32_t* in_nbr,
                                            int64_t node_capacity, int64_t edge_capacity,
                                            int64_t* num_nodes, int64_t* num_edges) {
  if (nrows < 0 || !num_nodes || !num_edges || !out_off || !in_off ||
      (nrows > 0 && (!src || !dst || !node_ids || !out_nbr || !in_nbr))) {
    set_error("ringo_table_to_graph_noalloc: bad argument (negative size or NULL pointer)");
    return RINGO_EINVAL;
  }
  if (nrows > (int64_t)kMaxRows) {
    set_error("ringo_table_to_graph_noalloc: nrows exceeds RINGO_NOALLOC_MAX_ROWS "
              "(the fixed scratch array holds tables of at most 1048576 rows)");
    return RINGO_ERANGE;
  }
  if (edge_capacity < nrows) {
    set_error("ringo_table_to_graph_noalloc: edge_capacity must be at least nrows");
    return RINGO_ERANGE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = nullptr;
  int rc = scratch_address(&ws);
  if (rc != RINGO_OK) return rc;
  *num_nodes = 0;
  *num_edges = 0;
#define NA_TRY(x)                                                              \
  do {                                                                         \
    cudaError_t _e = (x);                                                      \
    if (_e != cudaSuccess) {                                                   \
      set_error(std::string(#x) + ": " + cudaGetErrorString(_e));              \
      return RINGO_ECUDA;                                                      \
    }                                                                          \
  } while (0)
  if (nrows == 0) {
    NA_TRY(cudaMemsetAsync(out_off, 0, sizeof(int64_t), s));
    NA_TRY(cudaMemsetAsync(in_off, 0, sizeof(int64_t), s));
    NA_TRY(cudaStreamSynchronize(s));
    return RINGO_OK;
  }
  const uint32_t n = (uint32_t)nrows;
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
  Ctl* dctl = (Ctl*)(ws + kOffCtl);
  Ctl h;  // host staging copy of the control block (pageable, on the stack)
  memset(&h, 0, sizeof(h));
  h.n_rows = n;
  h.src = src;
  h.dst = dst;
  h.keysA = (uint64_t*)(ws + kOffKeysA);
  h.keysB = (uint64_t*)(ws + kOffKeysB);
  h.status[0] = (uint32_t*)(ws + kOffSt0);
  h.status[1] = (uint32_t*)(ws + kOffSt1);
  h.status_rows = tiles;
  const size_t chunks = (tiles + kChunkTiles - 1) / kChunkTiles;
  for (int r = 0; r < 2; ++r) place_radix_chunks(&h, r, ws + (r ? kOffCh1 : kOffCh0), chunks);
  h.chunk_rows = (uint32_t)chunks;
  place_scan(&h, 0, ws + kOffSc0, tiles);
  place_scan(&h, 1, ws + kOffSc1, tiles);
  place_scan(&h, 2, ws + kOffSc2, ((size_t)2 * n + kMergeTile - 1) / kMergeTile + 1);
  h.usrc = (int32_t*)(ws + kOffUsrc);
  h.usrc_start = (int32_t*)(ws + kOffUsrcStart);
  h.udst = (int32_t*)(ws + kOffUdst);
  h.udst_start = (int32_t*)(ws + kOffUdstStart);
  h.out_nbr = out_nbr;
  h.in_nbr = in_nbr;
  // state left by the previous call: the control block is rewritten whole,
  // status region 0 and the scan statuses are cleared
  Launch run = solo_launch(dctl, &h, n);
  run.opts = sort_opts_for(0, n);
  NA_TRY(cudaMemcpyAsync(dctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  NA_TRY(cudaMemsetAsync(ws + kOffSt0, 0, radix_status_bytes(tiles), s));
  NA_TRY(cudaMemsetAsync(ws + kOffCh0, 0, radix_chunk_bytes(chunks), s));
  NA_TRY(cudaMemsetAsync(ws + kOffSc0, 0, kOffUsrc - kOffSc0, s));
  if ((rc = enqueue_phase1(run, s)) != RINGO_OK) return rc;
  NA_TRY(cudaMemcpyAsync(&h, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
  if (h.err) {
    set_error("ringo_table_to_graph_noalloc: a bounded device wait expired");
    return RINGO_ETIMEOUT;
  }
  const uint64_t cap = (uint64_t)h.Vs + h.Vd;
  if ((int64_t)cap > node_capacity) {
    set_error("ringo_table_to_graph_noalloc: node_capacity is below (distinct sources + "
              "distinct destinations) of this table; 2 * nrows always suffices");
    return RINGO_ERANGE;
  }
  int32_t* ranks = (int32_t*)(ws + kOffRanks);
  h.node_ids = node_ids;
  h.out_off = out_off;
  h.in_off = in_off;
  h.src_rank = ranks;
  h.dst_rank = ranks + up4(h.Vs);
  h.src_blk = (uint32_t*)(h.dst_rank + up4(h.Vd));
  h.dst_blk = h.src_blk + up4((h.Vs + 31) / 32);
  NA_TRY(cudaMemcpyAsync(dctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  if ((rc = enqueue_phase2(run, s)) != RINGO_OK) return rc;
  if ((rc = enqueue_phase3(run, s)) != RINGO_OK) return rc;
  NA_TRY(cudaMemcpyAsync(&h, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
#undef NA_TRY
  if (h.err & (kErrLookback | kErrScan)) {
    set_error("ringo_table_to_graph_noalloc: a bounded device wait expired");
    return RINGO_ETIMEOUT;
  }
  if (h.err & kErrRemap) {
    set_error("ringo_table_to_graph_noalloc: internal error in the remap");
    return RINGO_ECUDA;
  }
  *num_nodes = h.V;
  *num_edges = h.E;
  return RINGO_OK;
}
