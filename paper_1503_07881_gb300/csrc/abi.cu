// C ABI of libringo (declared in include/ringo.h) and the host side of the
// table->graph conversion (paper, Section 3.4).  The kernel sequence itself
// is in pipeline.cu:
//   phase 1  histogram, 4 dst passes, dst ranks, 4 src passes, dedup
//   -- stream sync: E, Vs, Vd; node arrays and rank maps allocated --
//   phase 2  merge, block tables, out-direction remap: the out-CSR is done
//   phase 3  plan + 4 in-sort passes, destination runs (in_nbr), in_off
//   -- stream sync: V and the error word --
// With host outputs (ringo_table_to_graph_host_io) the out-CSR goes back to
// the host on a second stream while phase 3 runs.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <string>

#include "../../include/ringo.h"
#include "host_util.h"
#include "ringo_internal.cuh"

using namespace ringo;

struct ringo_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  ringo_graph_info info{};
  int32_t* node_ids = nullptr;
  int64_t* out_off = nullptr;
  int32_t* out_nbr = nullptr;
  int64_t* in_off = nullptr;
  int32_t* in_nbr = nullptr;
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

void free_graph_arrays(ringo_graph* g) {
  pool_free(g->node_ids, g->stream);
  pool_free(g->out_off, g->stream);
  pool_free(g->out_nbr, g->stream);
  pool_free(g->in_off, g->stream);
  pool_free(g->in_nbr, g->stream);
  g->node_ids = nullptr;
  g->out_off = g->in_off = nullptr;
  g->out_nbr = g->in_nbr = nullptr;
}

// Graph of an empty table: no nodes, no edges, offsets {0}.
int make_empty(ringo_graph* g) {
  g->out_off = (int64_t*)pool_alloc(sizeof(int64_t), g->stream);
  g->in_off = (int64_t*)pool_alloc(sizeof(int64_t), g->stream);
  if (!g->out_off || !g->in_off) return RINGO_ENOMEM;
  RINGO_CUDA_TRY(cudaMemsetAsync(g->out_off, 0, sizeof(int64_t), g->stream));
  RINGO_CUDA_TRY(cudaMemsetAsync(g->in_off, 0, sizeof(int64_t), g->stream));
  RINGO_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return RINGO_OK;
}

struct WsLayout {
  size_t ctl, keysA, keysB, st0, st1, ch0, ch1, sc0, sc1, sc2, usrc, usrc_start, udst, udst_start,
      total;
  size_t chunks, chunk_bytes;
};

size_t chunks_for(size_t tiles) { return (tiles + kChunkTiles - 1) / kChunkTiles; }
size_t scan_bytes(size_t tiles) {
  const size_t c = chunks_for(tiles);
  return align_up(8 * tiles) + align_up(8 * c) + align_up(8 * c) + align_up(4 * c);
}
void place_scan(Ctl* h, int i, char* p, size_t tiles) {
  const size_t c = chunks_for(tiles);
  h->scan_status[i] = (uint64_t*)p;
  p += align_up(8 * tiles);
  h->scan_chunk_agg[i] = (uint64_t*)p;
  p += align_up(8 * c);
  h->scan_chunk_inc[i] = (uint64_t*)p;
  p += align_up(8 * c);
  h->scan_chunk_cnt[i] = (uint32_t*)p;
}

WsLayout layout_for(uint32_t n) {
  const size_t tiles = (n + kSortTile - 1) / kSortTile;
  const size_t mtiles = ((size_t)2 * n + kMergeTile - 1) / kMergeTile + 1;
  WsLayout L{};
  size_t o = 0;
  L.ctl = o; o = align_up(o + sizeof(Ctl));
  L.keysA = o; o = align_up(o + sizeof(uint64_t) * ((size_t)n + 1));
  L.keysB = o; o = align_up(o + sizeof(uint64_t) * ((size_t)n + 1));
  L.st0 = o; o = align_up(o + radix_status_bytes(tiles));
  L.st1 = o; o = align_up(o + radix_status_bytes(tiles));
  L.chunks = (tiles + kChunkTiles - 1) / kChunkTiles;
  L.chunk_bytes = align_up(radix_chunk_bytes(L.chunks));
  L.ch0 = o; o = align_up(o + L.chunk_bytes);
  L.ch1 = o; o = align_up(o + L.chunk_bytes);
  // per scan: tile statuses, then chunk sums, chunk prefixes, chunk counters
  L.sc0 = o; o = align_up(o + scan_bytes(tiles));
  L.sc1 = o; o = align_up(o + scan_bytes(tiles));
  L.sc2 = o; o = align_up(o + scan_bytes(mtiles));
  L.usrc = o; o = align_up(o + sizeof(int32_t) * ((size_t)n + 1));
  L.usrc_start = o; o = align_up(o + sizeof(int32_t) * ((size_t)n + 1));
  L.udst = o; o = align_up(o + sizeof(int32_t) * ((size_t)n + 1));
  L.udst_start = o; o = align_up(o + sizeof(int32_t) * ((size_t)n + 1));
  L.total = o;
  return L;
}

// Words of the rank-map region: src_rank[Vs], dst_rank[Vd], and the two
// block tables, each part 16-byte aligned.
inline size_t up4(size_t x) { return (x + 3) & ~(size_t)3; }
inline size_t rank_region_words(uint32_t Vs, uint32_t Vd) {
  return up4(Vs) + up4(Vd) + up4((Vs + 31) / 32) + up4((Vd + 31) / 32);
}
void place_rank_region(Ctl* h, int32_t* base, uint32_t Vs, uint32_t Vd) {
  h->src_rank = base;
  h->dst_rank = base + up4(Vs);
  h->src_blk = (uint32_t*)(h->dst_rank + up4(Vd));
  h->dst_blk = h->src_blk + up4((Vs + 31) / 32);
}

// Caller-owned host arrays for the result (ringo_table_to_graph_host_io).
struct HostOut {
  int32_t* node_ids;
  int64_t* out_off;
  int32_t* out_nbr;
  int64_t* in_off;
  int32_t* in_nbr;
  int64_t node_capacity, edge_capacity;
};

// The conversion proper, for 1 <= n < 2^31 device rows.  With `ho`, the
// result is also copied into the caller's host arrays: the out-CSR on a
// second stream while phase 3 runs, the in-CSR after it.
int convert(const int32_t* d_src, const int32_t* d_dst, uint32_t n, ringo_graph* g,
            const HostOut* ho = nullptr) {
  cudaStream_t s = g->stream;
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
  const WsLayout L = layout_for(n);
  char* ws = (char*)pool_alloc(L.total, s);
  if (!ws) return RINGO_ENOMEM;
  g->out_nbr = (int32_t*)pool_alloc(sizeof(int32_t) * (size_t)n, s);
  g->in_nbr = (int32_t*)pool_alloc(sizeof(int32_t) * (size_t)n, s);
  Ctl* hctl = (Ctl*)pinned_get(sizeof(Ctl));
  int32_t* ranks = nullptr;
  int rc = RINGO_OK;
  Ctl* dctl = (Ctl*)(ws + L.ctl);
  cudaStream_t cs = nullptr;  // host outputs: the out-CSR's copy stream
  cudaEvent_t ev2 = nullptr;  // host outputs: phase 2 done
  if (ho && (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming) != cudaSuccess)) {
    set_error("copy stream or event creation failed");
    rc = RINGO_ECUDA;
    goto done;
  }
  if (!g->out_nbr || !g->in_nbr || !hctl) {
    rc = RINGO_ENOMEM;
    if (!hctl) set_error("pinned staging allocation failed");
    goto done;
  }
  {
    memset(hctl, 0, sizeof(Ctl));
    hctl->n_rows = n;
    hctl->src = d_src;
    hctl->dst = d_dst;
    hctl->keysA = (uint64_t*)(ws + L.keysA);
    hctl->keysB = (uint64_t*)(ws + L.keysB);
    hctl->status[0] = (uint32_t*)(ws + L.st0);
    hctl->status[1] = (uint32_t*)(ws + L.st1);
    hctl->status_rows = tiles;
    for (int r = 0; r < 2; ++r) place_radix_chunks(hctl, r, ws + (r ? L.ch1 : L.ch0), L.chunks);
    hctl->chunk_rows = (uint32_t)L.chunks;
    place_scan(hctl, 0, ws + L.sc0, tiles);
    place_scan(hctl, 1, ws + L.sc1, tiles);
    place_scan(hctl, 2, ws + L.sc2, ((size_t)2 * n + kMergeTile - 1) / kMergeTile + 1);
    hctl->usrc = (int32_t*)(ws + L.usrc);
    hctl->usrc_start = (int32_t*)(ws + L.usrc_start);
    hctl->udst = (int32_t*)(ws + L.udst);
    hctl->udst_start = (int32_t*)(ws + L.udst_start);
    hctl->out_nbr = g->out_nbr;
    hctl->in_nbr = g->in_nbr;
#define TRY(x)                         \
  do {                                 \
    cudaError_t _e = (x);              \
    if (_e != cudaSuccess) {           \
      set_error(std::string(#x) + ": " + cudaGetErrorString(_e)); \
      rc = RINGO_ECUDA;                \
      goto done;                       \
    }                                  \
  } while (0)
    Launch run = solo_launch(dctl, hctl, n);
    run.opts = sort_opts_for(0, n);
    if (const uint32_t lim = take_lookback_timeout()) {
      // failure-detection test: every wait of this conversion is bounded by
      // `lim` spins, and the first radix pass starts claiming at slot 1, so
      // its tile 0 is never processed and the tiles after it wait on it
      hctl->spin_limit = lim;
      hctl->solo_counters[1] = 1;
    }
    TRY(cudaMemcpyAsync(dctl, hctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    // status region 0 must start clear; each pass clears the other region
    TRY(cudaMemsetAsync(ws + L.st0, 0, L.st1 - L.st0, s));
    TRY(cudaMemsetAsync(ws + L.ch0, 0, L.chunk_bytes, s));
    TRY(cudaMemsetAsync(ws + L.sc0, 0, L.usrc - L.sc0, s));
    if ((rc = enqueue_phase1(run, s)) != RINGO_OK) goto done;
    TRY(cudaMemcpyAsync(hctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (hctl->err) {
      set_error("a bounded device wait expired during the sort");
      rc = RINGO_ETIMEOUT;
      goto done;
    }
    const uint64_t cap = (uint64_t)hctl->Vs + hctl->Vd;
    if (cap > 0x7FFFFFFFull) {
      set_error("node count does not fit int32");
      rc = RINGO_ERANGE;
      goto done;
    }
    g->node_ids = (int32_t*)pool_alloc(sizeof(int32_t) * cap, s);
    g->out_off = (int64_t*)pool_alloc(sizeof(int64_t) * (cap + 1), s);
    g->in_off = (int64_t*)pool_alloc(sizeof(int64_t) * (cap + 1), s);
    ranks = (int32_t*)pool_alloc(sizeof(int32_t) * rank_region_words(hctl->Vs, hctl->Vd), s);
    if (!g->node_ids || !g->out_off || !g->in_off || !ranks) {
      rc = RINGO_ENOMEM;
      goto done;
    }
    hctl->node_ids = g->node_ids;
    hctl->out_off = g->out_off;
    hctl->in_off = g->in_off;
    place_rank_region(hctl, ranks, hctl->Vs, hctl->Vd);
    TRY(cudaMemcpyAsync(dctl, hctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    if ((rc = enqueue_phase2(run, s)) != RINGO_OK) goto done;
    if (ho) {
      // V is known once phase 2 is done; the out-CSR can go back while the
      // in-sort runs
      if (hctl->E > ho->edge_capacity) {
        set_error("edge_capacity is below the number of distinct edges");
        rc = RINGO_ERANGE;
        goto done;
      }
      TRY(cudaMemcpyAsync(&hctl->V, &dctl->V, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      TRY(cudaEventRecord(ev2, s));
      if ((rc = enqueue_phase3(run, s)) != RINGO_OK) goto done;
      TRY(cudaEventSynchronize(ev2));
      const uint64_t V = hctl->V;
      if ((int64_t)V > ho->node_capacity) {
        set_error("node_capacity is below the number of nodes");
        rc = RINGO_ERANGE;
        goto done;
      }
      TRY(cudaStreamWaitEvent(cs, ev2, 0));
      {
        ProfScope ps("out_csr_d2h", cs);
        if (V) TRY(cudaMemcpyAsync(ho->node_ids, g->node_ids, 4 * V, cudaMemcpyDeviceToHost, cs));
        TRY(cudaMemcpyAsync(ho->out_off, g->out_off, 8 * (V + 1), cudaMemcpyDeviceToHost, cs));
        if (hctl->E)
          TRY(cudaMemcpyAsync(ho->out_nbr, g->out_nbr, 4ull * hctl->E, cudaMemcpyDeviceToHost,
                              cs));
      }
    } else {
      if ((rc = enqueue_phase3(run, s)) != RINGO_OK) goto done;
    }
    TRY(cudaMemcpyAsync(hctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (hctl->err & (kErrLookback | kErrScan)) {
      set_error("a bounded device wait expired");
      rc = RINGO_ETIMEOUT;
      goto done;
    }
    if (hctl->err & kErrRemap) {
      set_error("internal error in the run index -> node index remap");
      rc = RINGO_ECUDA;
      goto done;
    }
    g->info.nrows = n;
    g->info.num_nodes = hctl->V;
    g->info.num_edges = hctl->E;
    g->info.num_src_nodes = hctl->Vs;
    g->info.num_dst_nodes = hctl->Vd;
    g->info.out_sort_passes = (int32_t)hctl->out_sort.active_passes;
    g->info.in_sort_passes = (int32_t)hctl->in_sort.active_passes;
    if (ho) {
      const uint64_t V = hctl->V, E = hctl->E;
      ProfScope ps("in_csr_d2h", s);
      TRY(cudaMemcpyAsync(ho->in_off, g->in_off, 8 * (V + 1), cudaMemcpyDeviceToHost, s));
      if (E) TRY(cudaMemcpyAsync(ho->in_nbr, g->in_nbr, 4 * E, cudaMemcpyDeviceToHost, s));
    }
#undef TRY
  }
done:
  if (cs) {
    // the copy stream's work must be over before its buffers can go
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  if (ev2) cudaEventDestroy(ev2);
  if (ho && rc == RINGO_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("device->host copy: ") + cudaGetErrorString(cudaGetLastError()));
    rc = RINGO_ECUDA;
  }
  pool_free(ranks, s);
  pool_free(ws, s);
  if (hctl) pinned_put(hctl);
  return rc;
}

int check_dir(int dir) { return (dir == RINGO_OUT || dir == RINGO_IN) ? RINGO_OK : RINGO_EINVAL; }

}  // namespace

extern "C" {

const char* ringo_status_string(int status) {
  switch (status) {
    case RINGO_OK: return "ok";
    case RINGO_EINVAL: return "invalid argument";
    case RINGO_ENOMEM: return "out of memory";
    case RINGO_ECUDA: return "CUDA error";
    case RINGO_ETIMEOUT: return "device wait timed out";
    case RINGO_ENOTFOUND: return "not found";
    case RINGO_EBUSY: return "busy";
    case RINGO_ERANGE: return "size out of range";
    default: return "unknown status";
  }
}

const char* ringo_last_error(void) { return ringo::last_error(); }

const char* ringo_version(void) { return "ringo-gb300 0.1 sm_103a"; }

static int table_to_graph_impl(const int32_t* src, const int32_t* dst, int64_t nrows,
                               void* stream, ringo_graph** out, bool host) {
  if (!out) {
    set_error("out is NULL");
    return RINGO_EINVAL;
  }
  *out = nullptr;
  if (nrows < 0 || (nrows > 0 && (!src || !dst))) {
    set_error("nrows < 0 or NULL column");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF) {
    set_error("nrows exceeds 2^31 - 1");
    return RINGO_ERANGE;
  }
  ringo_graph* g = new (std::nothrow) ringo_graph();
  if (!g) return RINGO_ENOMEM;
  g->stream = (cudaStream_t)stream;
  cudaGetDevice(&g->device);
  int rc;
  if (nrows == 0) {
    rc = make_empty(g);
  } else if (host) {
    const size_t bytes = sizeof(int32_t) * (size_t)nrows;
    int32_t* d_src = nullptr;
    int32_t* d_dst = nullptr;
    {
      HostScope hs("host:input_alloc");
      d_src = (int32_t*)pool_alloc(bytes, g->stream);
      d_dst = (int32_t*)pool_alloc(bytes, g->stream);
    }
    bool copied = false;
    if (d_src && d_dst) {
      ProfScope ps("input_h2d", g->stream);
      copied = cudaMemcpyAsync(d_src, src, bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess &&
               cudaMemcpyAsync(d_dst, dst, bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess;
    }
    if (!d_src || !d_dst) {
      rc = RINGO_ENOMEM;
    } else if (!copied) {
      set_error(std::string("host->device copy failed: ") +
                cudaGetErrorString(cudaGetLastError()));
      rc = RINGO_ECUDA;
    } else {
      rc = convert(d_src, d_dst, (uint32_t)nrows, g);
    }
    pool_free(d_src, g->stream);
    pool_free(d_dst, g->stream);
  } else {
    rc = convert(src, dst, (uint32_t)nrows, g);
  }
  if (rc != RINGO_OK) {
    free_graph_arrays(g);
    delete g;
    return rc;
  }
  *out = g;
  return RINGO_OK;
}

int ringo_table_to_graph(const int32_t* src, const int32_t* dst, int64_t nrows, void* stream,
                         ringo_graph** out) {
  return table_to_graph_impl(src, dst, nrows, stream, out, false);
}

int ringo_table_to_graph_host(const int32_t* h_src, const int32_t* h_dst, int64_t nrows,
                              void* stream, ringo_graph** out) {
  return table_to_graph_impl(h_src, h_dst, nrows, stream, out, true);
}

int ringo_table_to_graph_host_io(const int32_t* h_src, const int32_t* h_dst, int64_t nrows,
                                 void* stream, int32_t* h_node_ids, int64_t* h_out_off,
                                 int32_t* h_out_nbr, int64_t* h_in_off, int32_t* h_in_nbr,
                                 int64_t node_capacity, int64_t edge_capacity,
                                 int64_t* num_nodes, int64_t* num_edges) {
  if (!num_nodes || !num_edges || !h_out_off || !h_in_off || nrows < 0 ||
      (nrows > 0 && (!h_src || !h_dst || !h_node_ids || !h_out_nbr || !h_in_nbr))) {
    set_error("ringo_table_to_graph_host_io: nrows < 0 or NULL pointer");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF) {
    set_error("nrows exceeds 2^31 - 1");
    return RINGO_ERANGE;
  }
  *num_nodes = 0;
  *num_edges = 0;
  if (nrows == 0) {
    h_out_off[0] = 0;
    h_in_off[0] = 0;
    return RINGO_OK;
  }
  ringo_graph* g = new (std::nothrow) ringo_graph();
  if (!g) return RINGO_ENOMEM;
  g->stream = (cudaStream_t)stream;
  cudaGetDevice(&g->device);
  const size_t bytes = sizeof(int32_t) * (size_t)nrows;
  int32_t* d_src = nullptr;
  int32_t* d_dst = nullptr;
  {
    HostScope hs("host:input_alloc");
    d_src = (int32_t*)pool_alloc(bytes, g->stream);
    d_dst = d_src ? (int32_t*)pool_alloc(bytes, g->stream) : nullptr;
  }
  int rc = RINGO_OK;
  if (!d_src || !d_dst) {
    rc = RINGO_ENOMEM;
  } else {
    bool copied;
    {
      ProfScope ps("input_h2d", g->stream);
      copied = cudaMemcpyAsync(d_src, h_src, bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess &&
               cudaMemcpyAsync(d_dst, h_dst, bytes, cudaMemcpyHostToDevice, g->stream) ==
                   cudaSuccess;
    }
    if (!copied) {
      set_error(std::string("host->device copy failed: ") +
                cudaGetErrorString(cudaGetLastError()));
      rc = RINGO_ECUDA;
    } else {
      const HostOut ho{h_node_ids, h_out_off, h_out_nbr, h_in_off, h_in_nbr, node_capacity,
                       edge_capacity};
      rc = convert(d_src, d_dst, (uint32_t)nrows, g, &ho);
    }
  }
  pool_free(d_src, g->stream);
  pool_free(d_dst, g->stream);
  if (rc == RINGO_OK) {
    *num_nodes = g->info.num_nodes;
    *num_edges = g->info.num_edges;
  }
  free_graph_arrays(g);
  delete g;
  return rc;
}

int ringo_table_to_undirected_graph(const int32_t* src, const int32_t* dst, int64_t nrows,
                                    void* stream, ringo_graph** out) {
  if (!out) return RINGO_EINVAL;
  *out = nullptr;
  if (nrows < 0 || (nrows > 0 && (!src || !dst))) {
    set_error("nrows < 0 or NULL column");
    return RINGO_EINVAL;
  }
  if (nrows > 0x7FFFFFFF) {
    set_error("nrows exceeds 2^31 - 1");
    return RINGO_ERANGE;
  }
  ringo_graph* g = new (std::nothrow) ringo_graph();
  if (!g) return RINGO_ENOMEM;
  g->stream = (cudaStream_t)stream;
  cudaGetDevice(&g->device);
  int rc;
  if (nrows == 0) {
    rc = make_empty(g);
  } else {
    // the directed graph, then each node's out- and in-list merged
    ringo_graph* d = new (std::nothrow) ringo_graph();
    if (!d) {
      rc = RINGO_ENOMEM;
    } else {
      d->stream = g->stream;
      d->device = g->device;
      rc = convert(src, dst, (uint32_t)nrows, d);
      int64_t* uoff = nullptr;
      int32_t* unbr = nullptr;
      uint64_t M = 0;
      if (rc == RINGO_OK)
        rc = build_undirected(d->out_off, d->out_nbr, d->in_off, d->in_nbr,
                              (uint32_t)d->info.num_nodes, (uint64_t)d->info.num_edges, g->stream,
                              &uoff, &unbr, &M);
      if (rc == RINGO_OK) {
        const uint64_t V = (uint64_t)d->info.num_nodes;
        g->info = d->info;
        g->info.num_edges = (int64_t)M;
        g->info.num_src_nodes = (int64_t)V;
        g->info.num_dst_nodes = (int64_t)V;
        g->node_ids = d->node_ids;  // the node list is the directed graph's
        d->node_ids = nullptr;
        g->out_off = uoff;
        g->out_nbr = unbr;
        // the in-CSR holds the same symmetric lists
        g->in_off = (int64_t*)pool_alloc(8 * (V + 1), g->stream);
        g->in_nbr = (int32_t*)pool_alloc(4 * M + 4, g->stream);
        if (!g->in_off || !g->in_nbr) {
          set_error("undirected: device memory for the in-direction copy");
          rc = RINGO_ENOMEM;
        } else if (cudaMemcpyAsync(g->in_off, uoff, 8 * (V + 1), cudaMemcpyDeviceToDevice,
                                   g->stream) != cudaSuccess ||
                   cudaMemcpyAsync(g->in_nbr, unbr, 4 * M, cudaMemcpyDeviceToDevice,
                                   g->stream) != cudaSuccess ||
                   cudaStreamSynchronize(g->stream) != cudaSuccess) {
          set_error(std::string("undirected copy: ") + cudaGetErrorString(cudaGetLastError()));
          rc = RINGO_ECUDA;
        }
      }
      free_graph_arrays(d);
      delete d;
    }
  }
  if (rc != RINGO_OK) {
    free_graph_arrays(g);
    delete g;
    return rc;
  }
  *out = g;
  return RINGO_OK;
}

int ringo_graph_count_triangles(const ringo_graph* g, void* stream, uint64_t* count) {
  if (!g || !count) return RINGO_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  return run_triangles(g->out_off, g->out_nbr, (uint32_t)g->info.num_nodes,
                       (uint64_t)g->info.num_edges, s, count);
}

int ringo_graph_num_nodes(const ringo_graph* g, int64_t* v) {
  if (!g || !v) return RINGO_EINVAL;
  *v = g->info.num_nodes;
  return RINGO_OK;
}

int ringo_graph_num_edges(const ringo_graph* g, int64_t* e) {
  if (!g || !e) return RINGO_EINVAL;
  *e = g->info.num_edges;
  return RINGO_OK;
}

int ringo_graph_get_info(const ringo_graph* g, ringo_graph_info* info) {
  if (!g || !info) return RINGO_EINVAL;
  *info = g->info;
  return RINGO_OK;
}

int ringo_graph_node_ids(const ringo_graph* g, const int32_t** d_ids) {
  if (!g || !d_ids) return RINGO_EINVAL;
  *d_ids = g->info.num_nodes ? g->node_ids : nullptr;
  return RINGO_OK;
}

int ringo_graph_csr(const ringo_graph* g, int dir, const int64_t** d_off, const int32_t** d_nbr) {
  if (!g || !d_off || !d_nbr || check_dir(dir)) return RINGO_EINVAL;
  *d_off = dir == RINGO_OUT ? g->out_off : g->in_off;
  *d_nbr = g->info.num_edges ? (dir == RINGO_OUT ? g->out_nbr : g->in_nbr) : nullptr;
  return RINGO_OK;
}

int ringo_graph_degrees(const ringo_graph* g, int dir, const int32_t* d_ids, int64_t n,
                        int64_t* d_deg, void* stream) {
  if (!g || check_dir(dir) || n < 0 || (n > 0 && (!d_ids || !d_deg))) return RINGO_EINVAL;
  if (n > 0x7FFFFFFF) return RINGO_ERANGE;
  if (n == 0) return RINGO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (g->info.num_nodes == 0) {
    RINGO_CUDA_TRY(cudaMemsetAsync(d_deg, 0xFF, sizeof(int64_t) * (size_t)n, s));
    return RINGO_OK;
  }
  {
    ProfScope ps("degrees", s);
    launch_degrees(g->node_ids, dir == RINGO_OUT ? g->out_off : g->in_off,
                   (uint32_t)g->info.num_nodes, d_ids, (uint32_t)n, d_deg, s);
  }
  RINGO_LAUNCH_CHECK("degrees");
  return RINGO_OK;
}

int ringo_graph_degree(const ringo_graph* g, int dir, int32_t node_id, int64_t* deg) {
  if (!g || !deg || check_dir(dir)) return RINGO_EINVAL;
  cudaStream_t s = g->stream;
  void* buf = pool_alloc(16, s);
  if (!buf) return RINGO_ENOMEM;
  int64_t* hbuf = (int64_t*)pinned_get(16);
  int rc = RINGO_OK;
  if (!hbuf) {
    pool_free(buf, s);
    return RINGO_ENOMEM;
  }
  hbuf[0] = node_id;
  int32_t* d_id = (int32_t*)buf;
  int64_t* d_deg = (int64_t*)((char*)buf + 8);
  if (cudaMemcpyAsync(d_id, hbuf, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    rc = RINGO_ECUDA;
  } else if ((rc = ringo_graph_degrees(g, dir, d_id, 1, d_deg, s)) == RINGO_OK) {
    if (cudaMemcpyAsync(hbuf + 1, d_deg, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = RINGO_ECUDA;
    } else if (hbuf[1] < 0) {
      rc = RINGO_ENOTFOUND;
    } else {
      *deg = hbuf[1];
    }
  }
  pool_free(buf, s);
  pinned_put(hbuf);
  return rc;
}

int ringo_graph_degree_topk(const ringo_graph* g, int dir, int32_t k, int32_t* h_ids,
                            int64_t* h_degs, int32_t* n_out) {
  if (!g || !n_out || check_dir(dir) || k < 0) return RINGO_EINVAL;
  if (k > 4096) {
    set_error("k above 4096");
    return RINGO_ERANGE;
  }
  const int64_t V = g->info.num_nodes;
  const uint32_t kk = (uint32_t)(k < V ? k : V);
  *n_out = (int32_t)kk;
  if (kk == 0) return RINGO_OK;
  if (!h_ids || !h_degs) return RINGO_EINVAL;
  cudaStream_t s = g->stream;
  const size_t sb = topk_scratch_bytes((uint32_t)V, kk);
  const size_t out_bytes = align_up(sizeof(int32_t) * kk) + sizeof(int64_t) * kk;
  char* buf = (char*)pool_alloc(align_up(sb) + out_bytes, s);
  if (!buf) return RINGO_ENOMEM;
  int32_t* d_ids = (int32_t*)(buf + align_up(sb));
  int64_t* d_degs = (int64_t*)(buf + align_up(sb) + align_up(sizeof(int32_t) * kk));
  int rc = RINGO_OK;
  {
    ProfScope ps("topk", s);
    if (launch_topk(g->node_ids, dir == RINGO_OUT ? g->out_off : g->in_off, (uint32_t)V, kk,
                    d_ids, d_degs, buf, sb, s) != 0)
      rc = RINGO_EINVAL;
  }
  if (rc == RINGO_OK) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_ids, d_ids, sizeof(int32_t) * kk, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_degs, d_degs, sizeof(int64_t) * kk, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("topk: ") + cudaGetErrorString(e));
      rc = RINGO_ECUDA;
    }
  }
  pool_free(buf, s);
  return rc;
}

int ringo_graph_copy_to_host(const ringo_graph* g, int32_t* h_node_ids, int64_t* h_out_off,
                             int32_t* h_out_nbr, int64_t* h_in_off, int32_t* h_in_nbr) {
  if (!g) return RINGO_EINVAL;
  cudaStream_t s = g->stream;
  const size_t V = (size_t)g->info.num_nodes, E = (size_t)g->info.num_edges;
  if (h_node_ids && V)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_node_ids, g->node_ids, 4 * V, cudaMemcpyDeviceToHost, s));
  if (h_out_off)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_out_off, g->out_off, 8 * (V + 1), cudaMemcpyDeviceToHost, s));
  if (h_out_nbr && E)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_out_nbr, g->out_nbr, 4 * E, cudaMemcpyDeviceToHost, s));
  if (h_in_off)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_in_off, g->in_off, 8 * (V + 1), cudaMemcpyDeviceToHost, s));
  if (h_in_nbr && E)
    RINGO_CUDA_TRY(cudaMemcpyAsync(h_in_nbr, g->in_nbr, 4 * E, cudaMemcpyDeviceToHost, s));
  RINGO_CUDA_TRY(cudaStreamSynchronize(s));
  return RINGO_OK;
}

int ringo_graph_to_edge_table(const ringo_graph* g, int dir, int32_t* d_src, int32_t* d_dst,
                              int64_t cap, int64_t* n, void* stream) {
  if (!g || !n || check_dir(dir) || cap < 0) return RINGO_EINVAL;
  const int64_t E = g->info.num_edges;
  *n = E;
  if (E > cap) {
    set_error("ringo_graph_to_edge_table: the graph has more edges than cap");
    return RINGO_ERANGE;
  }
  if (E && (!d_src || !d_dst)) return RINGO_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  const uint32_t V = (uint32_t)g->info.num_nodes;
  // out-CSR rows are (src, dst); in-CSR rows are (dst, src), swapped back
  if (dir == RINGO_OUT)
    return launch_edge_table(g->node_ids, g->out_off, g->out_nbr, V, (uint64_t)E, d_src, d_dst, s);
  return launch_edge_table(g->node_ids, g->in_off, g->in_nbr, V, (uint64_t)E, d_dst, d_src, s);
}

int ringo_graph_to_node_table(const ringo_graph* g, int32_t* d_ids, int64_t* d_outdeg,
                              int64_t* d_indeg, int64_t cap, int64_t* n, void* stream) {
  if (!g || !n || cap < 0) return RINGO_EINVAL;
  const int64_t V = g->info.num_nodes;
  *n = V;
  if (V > cap) {
    set_error("ringo_graph_to_node_table: the graph has more nodes than cap");
    return RINGO_ERANGE;
  }
  if (V && (!d_ids || !d_outdeg || !d_indeg)) return RINGO_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  return launch_node_table(g->node_ids, g->out_off, g->in_off, (uint32_t)V, d_ids, d_outdeg,
                           d_indeg, s);
}

int ringo_graph_pagerank(const ringo_graph* g, double damping, int32_t iterations, double* d_rank,
                         void* stream) {
  if (!g || iterations < 0 || !(damping >= 0.0 && damping <= 1.0)) return RINGO_EINVAL;
  const int64_t V = g->info.num_nodes, E = g->info.num_edges;
  if (V && !d_rank) return RINGO_EINVAL;
  cudaStream_t s = stream ? (cudaStream_t)stream : g->stream;
  return run_pagerank(g->out_off, g->in_off, g->in_nbr, (uint32_t)V, (uint64_t)E, damping,
                      iterations, d_rank, s);
}

void ringo_graph_free(ringo_graph* g) {
  if (!g) return;
  free_graph_arrays(g);
  delete g;
}

}  // extern "C"
