/*
 * ringo.h -- C ABI of the GB300 table->graph conversion library (libringo.so).
 *
 * The operation (paper, Section 3.4 "Conversion of tables to graphs"): given
 * an edge table T with a source column S and a destination column D, build
 * the directed graph G = (V, E) whose nodes are the unique values of S and D
 * and whose edges are the rows (r_S, r_D).  Like the paper's graph object
 * (Section 3.2 "Ringo graph representation"), every node keeps a sorted
 * vector of out-neighbours and a sorted vector of in-neighbours.
 *
 * Result layout (all device memory owned by the graph handle):
 *   node_ids[V]      int32, the distinct IDs of S and D in ascending signed
 *                    order; a node's INDEX is its position here.
 *   out_off[V+1]     int64 offsets; the out-neighbours of node r are
 *   out_nbr[E]       int32 node indices out_nbr[out_off[r] .. out_off[r+1]),
 *                    strictly increasing.
 *   in_off[V+1]      the same for in-neighbours.
 *   in_nbr[E]
 * Readings of the paper applied (it is silent on them): duplicate rows
 * collapse to one edge, self-loops are kept, neighbours are stored as node
 * indices (node_ids[nbr] gives the ID), offsets are int64.
 *
 * Conventions for every call:
 *   - The return value is a ringo_status; no call aborts the process.
 *     ringo_last_error() gives a message for the calling thread's last error.
 *   - Device pointers are plain CUDA device addresses of the current device.
 *     `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Input buffers are borrowed for the duration of the call only.
 *   - Pointers returned by the accessors are borrowed: they stay valid until
 *     ringo_graph_free() of their graph.
 *   - Limits: 0 <= nrows <= 2^31 - 1, and the node count must fit in int32
 *     (RINGO_ERANGE otherwise).  nrows == 0 is valid and gives V = E = 0 with
 *     each offset array equal to {0}.
 */
#ifndef RINGO_H_
#define RINGO_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RINGO_API __attribute__((visibility("default")))
#else
#define RINGO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RINGO_OK = 0,
  RINGO_EINVAL = 1,    /* bad argument: negative size, NULL pointer, bad enum */
  RINGO_ENOMEM = 2,    /* device or pinned-host allocation failed */
  RINGO_ECUDA = 3,     /* a CUDA runtime call failed (message in ringo_last_error) */
  RINGO_ETIMEOUT = 4,  /* a bounded device-side wait gave up; the result is invalid */
  RINGO_ENOTFOUND = 5, /* the queried node ID is not in the graph */
  RINGO_EBUSY = 6,     /* resource in use (server / batch slots) */
  RINGO_ERANGE = 7     /* size beyond the limits above */
} ringo_status;

typedef enum { RINGO_OUT = 0, RINGO_IN = 1 } ringo_dir;

typedef struct ringo_graph ringo_graph;

/* Sizes and pass counts of a built graph (for measurement and tests). */
typedef struct {
  int64_t nrows;          /* input rows N */
  int64_t num_nodes;      /* V */
  int64_t num_edges;      /* E: distinct (src, dst) pairs */
  int64_t num_src_nodes;  /* distinct IDs in the source column */
  int64_t num_dst_nodes;  /* distinct IDs in the destination column */
  int32_t out_sort_passes;/* radix passes that moved (src,dst) keys (of 8) */
  int32_t in_sort_passes; /* radix passes that moved (dst,src) keys (of 4) */
} ringo_graph_info;

RINGO_API const char* ringo_status_string(int status);
RINGO_API const char* ringo_last_error(void);
/* Library version string, e.g. "ringo-gb300 0.1 sm_103a". */
RINGO_API const char* ringo_version(void);

/*
 * ringo_table_to_graph -- Section 3.4: table (S, D) -> directed graph.
 *   src, dst  device int32 columns of nrows entries each (borrowed; any
 *             alignment; IDs may be any int32 value, duplicates and
 *             self-loops allowed).
 *   stream    cudaStream_t the work is ordered on.
 *   out       receives a new graph handle (caller frees with ringo_graph_free).
 * Blocks the calling thread until the graph is complete (it synchronises the
 * stream twice: once to size the node arrays, once at the end).
 * Errors: EINVAL (NULL out, nrows < 0, NULL column with nrows > 0), ERANGE,
 * ENOMEM, ECUDA, ETIMEOUT.  On error *out is set to NULL.
 */
RINGO_API int ringo_table_to_graph(const int32_t* src, const int32_t* dst, int64_t nrows,
                         void* stream, ringo_graph** out);

/*
 * ringo_table_to_graph_host -- the same conversion from HOST columns: the
 * columns are copied to the device on `stream` first (pinned host memory
 * gives full copy speed; pageable memory works but is staged by CUDA).
 */
RINGO_API int ringo_table_to_graph_host(const int32_t* h_src, const int32_t* h_dst, int64_t nrows,
                              void* stream, ringo_graph** out);

/*
 * ringo_table_to_graph_host_io -- Section 3.4 conversion from host columns
 * to host arrays in one call, for callers whose table and result live in
 * host memory: the columns go up, the graph is built on the device, and the
 * five arrays come back into caller-owned host buffers (layout as
 * ringo_graph_copy_to_host).  The out-CSR (node_ids, out_off, out_nbr) is
 * final before the in-sort starts and is copied back on a second stream
 * while the in-CSR is built; in_off and in_nbr follow.  Pinned host buffers
 * (cudaHostAlloc or registered) let the copies run at the link's rate and
 * overlap the kernels; pageable ones work but serialise.
 *   h_src, h_dst      host columns of nrows int32 IDs (borrowed for the call)
 *   h_node_ids        node_capacity entries   } caller-owned outputs;
 *   h_out_off, h_in_off  node_capacity + 1    } 2 * nrows nodes and nrows
 *   h_out_nbr, h_in_nbr  edge_capacity        } edges always suffice
 *   num_nodes, num_edges  host outputs: V and E
 * Errors: EINVAL (NULL pointer, nrows < 0), ERANGE (nrows >= 2^31, or a
 * capacity below V or E: found during the call, nothing of the graph is
 * copied then), ENOMEM, ECUDA, ETIMEOUT.  Device memory is allocated for
 * the call's duration only and freed before it returns.  Blocks.
 */
RINGO_API int ringo_table_to_graph_host_io(const int32_t* h_src, const int32_t* h_dst,
                                           int64_t nrows, void* stream, int32_t* h_node_ids,
                                           int64_t* h_out_off, int32_t* h_out_nbr,
                                           int64_t* h_in_off, int32_t* h_in_nbr,
                                           int64_t node_capacity, int64_t edge_capacity,
                                           int64_t* num_nodes, int64_t* num_edges);

RINGO_API int ringo_graph_num_nodes(const ringo_graph* g, int64_t* v);
RINGO_API int ringo_graph_num_edges(const ringo_graph* g, int64_t* e);
RINGO_API int ringo_graph_get_info(const ringo_graph* g, ringo_graph_info* info);

/* Borrowed device pointer to node_ids[V] (NULL when V == 0). */
RINGO_API int ringo_graph_node_ids(const ringo_graph* g, const int32_t** d_ids);

/* Borrowed device pointers to one direction's CSR: off[V+1], nbr[E]. */
RINGO_API int ringo_graph_csr(const ringo_graph* g, int dir, const int64_t** d_off,
                    const int32_t** d_nbr);

/*
 * ringo_graph_degree -- out- or in-degree of one node given by its ID
 * (a binary search of node_ids on the device).  ENOTFOUND if absent.
 */
RINGO_API int ringo_graph_degree(const ringo_graph* g, int dir, int32_t node_id, int64_t* deg);

/*
 * ringo_graph_degrees -- batched degree query on the device:
 *   d_ids[n] node IDs (device), d_deg[n] (device, written): the degree, or -1
 *   for an ID that is not a node.  Ordered on `stream`; does not block.
 */
RINGO_API int ringo_graph_degrees(const ringo_graph* g, int dir, const int32_t* d_ids, int64_t n,
                        int64_t* d_deg, void* stream);

/*
 * ringo_graph_degree_topk -- the k nodes of largest degree in direction
 * `dir`, ordered by degree descending then node ID ascending.
 *   h_ids[k], h_degs[k]  host output arrays (caller-owned)
 *   n_out                number written: min(k, V)
 * 0 <= k <= 4096, else ERANGE.
 */
RINGO_API int ringo_graph_degree_topk(const ringo_graph* g, int dir, int32_t k, int32_t* h_ids,
                            int64_t* h_degs, int32_t* n_out);

/*
 * ringo_graph_copy_to_host -- copy all five arrays into caller-owned host
 * buffers sized V, V+1, E, V+1, E.  Any pointer may be NULL to skip that
 * array.  Blocks until the copies are done.
 */
RINGO_API int ringo_graph_copy_to_host(const ringo_graph* g, int32_t* h_node_ids, int64_t* h_out_off,
                             int32_t* h_out_nbr, int64_t* h_in_off, int32_t* h_in_nbr);

/* Release the graph and its device memory (NULL is a no-op). */
RINGO_API void ringo_graph_free(ringo_graph* g);

/*
 * ringo_table_to_graph_noalloc -- the same conversion for callers that cannot
 * allocate device memory at the time of the call (a fixed memory budget
 * reserved up front, a serving loop that must not enter the allocator).
 * The paper has no counterpart: this is a property of this library only.
 *   The call allocates no device or pinned host memory.  Scratch space is
 *   one fixed __device__ array inside the library (43.4 MB = 41.4 MiB per GPU, held
 *   until the process exits), so:
 *   - nrows <= RINGO_NOALLOC_MAX_ROWS, else RINGO_ERANGE;
 *   - calls whose GPU work overlaps (other streams or threads) race on that
 *     array and give wrong results: callers serialise them;
 *   - the array is placed on a GPU when the library's device code is loaded
 *     there, which (CUDA's lazy module loading being the default) is the
 *     first call on that device: that call looks up the array's address,
 *     takes the array's device memory, and returns RINGO_ENOMEM if there is
 *     none left.  Make the first call per device at set-up time.
 *   - the call blocks (two stream synchronisations, sizes read back in
 *     between), so it cannot be used inside a stream capture.
 *   src, dst          device columns of nrows int32 IDs (borrowed)
 *   node_ids          device, node_capacity entries       } caller-owned
 *   out_off, in_off   device, node_capacity + 1 entries   } outputs, same
 *   out_nbr, in_nbr   device, edge_capacity entries       } layout as above
 *   edge_capacity     must be >= nrows
 *   node_capacity     must be >= distinct sources + distinct destinations of
 *                     the table (2 * nrows always suffices), else RINGO_ERANGE
 *   num_nodes, num_edges  host outputs: V and E
 * Returns once the result is complete.  A node_capacity that turns out too
 * small is found after the sort (RINGO_ERANGE); the call has then written
 * out_nbr, in_nbr and the scratch array, and the next call is unaffected.
 */
#define RINGO_NOALLOC_MAX_ROWS (1 << 20)
RINGO_API int ringo_table_to_graph_noalloc(const int32_t* src, const int32_t* dst, int64_t nrows,
                                           void* stream, int32_t* node_ids, int64_t* out_off,
                                           int32_t* out_nbr, int64_t* in_off, int32_t* in_nbr,
                                           int64_t node_capacity, int64_t edge_capacity,
                                           int64_t* num_nodes, int64_t* num_edges);

/*
 * ringo_graph_to_edge_table -- Section 3.4 "Conversion of graphs to tables":
 * the graph's edge table, one row per edge, written to caller-owned device
 * columns d_src[cap], d_dst[cap] (node IDs).  dir RINGO_OUT gives the rows in
 * out-CSR order (sources ascending, each source's destinations ascending),
 * RINGO_IN in in-CSR order (destinations ascending, then sources); either
 * converts back to the same graph.  *n receives E.  Enqueued on `stream`
 * (NULL: the graph's stream); the columns are complete when the stream
 * reaches this point.  Errors: EINVAL (NULL g or n, bad dir, cap < 0, NULL
 * column with E > 0), ERANGE (cap < E; nothing written), ECUDA.
 */
RINGO_API int ringo_graph_to_edge_table(const ringo_graph* g, int dir, int32_t* d_src,
                                        int32_t* d_dst, int64_t cap, int64_t* n, void* stream);
/*
 * ringo_graph_to_node_table -- the node table: one row per node in ascending
 * ID order, with its out- and in-degree, into caller-owned device columns
 * d_ids[cap], d_outdeg[cap], d_indeg[cap].  *n receives V.  Stream and errors
 * as ringo_graph_to_edge_table (ERANGE if cap < V).
 */
RINGO_API int ringo_graph_to_node_table(const ringo_graph* g, int32_t* d_ids, int64_t* d_outdeg,
                                        int64_t* d_indeg, int64_t cap, int64_t* n, void* stream);

/*
 * ringo_graph_pagerank -- PageRank of the graph, the paper's second workload
 * (Section 4, Table "paralg": ten iterations).  Power iteration from the
 * uniform vector, in fp64:
 *   PR'(v) = (1 - d) / V + d * (sum over in-neighbours u of PR(u) / outdeg(u)
 *                               + sum of PR over nodes without out-edges / V),
 * `iterations` steps (0 gives the uniform vector), d = damping in [0, 1].
 * Writes PR in node-index order to caller-owned device d_rank[V].  Enqueued
 * on `stream` (NULL: the graph's stream); scratch of about 24 V + E / 85
 * bytes comes from the library's pool.  PR(u) / outdeg(u) is computed as
 * PR(u) * (1 / outdeg(u)) with the reciprocal formed once.  Each node's sum
 * is formed in a fixed order (the in-edges cut into 2048-edge tiles: runs of
 * 8 edges per thread, a scan over the tile's threads, then the node's tile
 * shares in tile order), so runs agree bit for bit; a sequential loop sums
 * in another order and agrees to within fp64 rounding (about max in-degree
 * x 1e-16 relative per step).
 * Errors: EINVAL (NULL g, NULL d_rank with V > 0, iterations < 0, damping
 * outside [0, 1]), ENOMEM, ECUDA.
 */
RINGO_API int ringo_graph_pagerank(const ringo_graph* g, double damping, int32_t iterations,
                                   double* d_rank, void* stream);

/*
 * ringo_table_to_undirected_graph -- the undirected graph of an edge table,
 * for the paper's undirected workload (Section 4, triangle counting): each
 * row (s, d) is the edge {s, d}; every distinct pair is one edge; a node's
 * list holds each neighbour once, sorted (node indices); a self-loop puts the
 * node once in its own list.  Both CSR directions hold the same symmetric
 * lists (num_edges counts each non-loop edge twice, once per endpoint).  The
 * table goes through ringo_table_to_graph's conversion and each node's out-
 * and in-list are then merged, so nrows is at most 2^31 - 1 (ERANGE above)
 * and the device memory needed is that of the directed graph plus the
 * undirected lists (twice, one per CSR direction).  The node list and
 * num_src_nodes = num_dst_nodes = V describe the undirected graph; the sort
 * pass counts are the directed conversion's.  Arguments and other errors as
 * ringo_table_to_graph.
 */
RINGO_API int ringo_table_to_undirected_graph(const int32_t* src, const int32_t* dst,
                                              int64_t nrows, void* stream, ringo_graph** out);
/*
 * ringo_graph_count_triangles -- the number of triangles (three distinct
 * nodes, each pair joined) of the undirected graph held in g's out-CSR, which
 * must be symmetric (as built by ringo_table_to_undirected_graph); self-loops
 * are ignored.  Exact (64-bit integer).  Scratch of about 22 V + 6 E bytes
 * from the library's pool (E = num_edges, the adjacency entries); blocks
 * until *count is on the host.
 * Errors: EINVAL (NULL g or count), ENOMEM, ECUDA.
 */
RINGO_API int ringo_graph_count_triangles(const ringo_graph* g, void* stream, uint64_t* count);

/* ------------------------------------------------------------------------
 * Select and join on edge tables: the relational operations that build the
 * edge table before conversion (Section 3.3, "Tables in Ringo"; Section 4,
 * Table "table_ringo").  Both keep row order and are enqueued on `stream`;
 * they block until the output row count is on the host.
 * ---------------------------------------------------------------------- */
typedef enum {
  RINGO_CMP_LT = 0, RINGO_CMP_LE = 1, RINGO_CMP_EQ = 2,
  RINGO_CMP_NE = 3, RINGO_CMP_GE = 4, RINGO_CMP_GT = 5
} ringo_cmp;

/*
 * ringo_table_select -- select in place: keeps the rows of the edge table
 * (device columns src, dst of nrows entries, caller-owned) whose column
 * `col` (0: src, 1: dst) compares with `value` by `op`, in their order, in
 * the first *n_out rows of both columns (the rest is left unspecified).
 * Errors: EINVAL (NULL n_out, NULL column with nrows > 0, nrows < 0, bad col
 * or op), ERANGE (nrows >= 2^31), ENOMEM, ETIMEOUT, ECUDA.
 */
RINGO_API int ringo_table_select(int32_t* src, int32_t* dst, int64_t nrows, int col, int op,
                                 int32_t value, int64_t* n_out, void* stream);
/*
 * ringo_table_join -- equi-join of the edge table with a single-column table
 * keys[nkeys] (device) on column `col`: every row whose key occurs in keys,
 * once per occurrence, in row order, written to caller-owned device columns
 * out_src[cap], out_dst[cap].  *n_out receives the join's row count; if it
 * exceeds cap (or 2^31 - 1) nothing is written and ERANGE is returned.
 * Device scratch during the call: 2 bits per row of the table, and the key
 * set: an open-addressing table of 16 to 32 bytes per key, or, when
 * smaller, two bitmaps over the keys' value range (at most 1 GB, for keys
 * spanning the whole int32 range) plus a table of the repeated keys.
 * Errors: EINVAL (bad pointers, sizes or col), ERANGE (nrows >= 2^31,
 * nkeys >= 2^30, output above cap), ENOMEM, ETIMEOUT, ECUDA.
 */
RINGO_API int ringo_table_join(const int32_t* src, const int32_t* dst, int64_t nrows, int col,
                               const int32_t* keys, int64_t nkeys, int32_t* out_src,
                               int32_t* out_dst, int64_t cap, int64_t* n_out, void* stream);

/* ------------------------------------------------------------------------
 * Base tables, selection and batched conversion.
 *
 * The paper builds graphs from tables after relational operations such as
 * select (Section 3.3 "Tables in Ringo"; rows keep persistent IDs there so
 * that selections can work in place).  A base table of edge rows with a
 * timestamp and a tag is loaded once and kept resident on the device,
 * clustered by (tag, ts); a predicate (a set of tags and a time window)
 * selects a sub-table, and a batch converts many selected sub-tables
 * (Section 3.4) at once, every kernel running over all of them.
 * ---------------------------------------------------------------------- */
typedef struct ringo_base ringo_base;
typedef struct ringo_batch ringo_batch;

/* A predicate: the rows with tag in tags[0 .. ntags) and t0 <= ts < t1.
 * tags is a caller-owned host array read during the call only; a repeated
 * value counts once; ntags == 0 or t1 <= t0 selects nothing. */
typedef struct {
  const int32_t* tags;
  int32_t ntags;
  int64_t t0;
  int64_t t1;
} ringo_select;

/*
 * ringo_base_table_load -- copy a base table of nrows rows from device
 * columns src, dst (int32 node IDs), ts (int64) and tag (int32), all of
 * length nrows and caller-owned, into library-owned device memory clustered
 * by (tag, ts) (two stable radix sorts; equal keys keep their row order).
 * The caller's columns are only read and may be freed on return.  Blocks
 * until done; *out owns the copy until ringo_base_table_free.
 * Errors: EINVAL (NULL out, nrows < 0, NULL column with nrows > 0), ERANGE
 * (nrows >= 2^31, or max(ts) - min(ts) >= 2^32), ENOMEM, ECUDA.
 */
RINGO_API int ringo_base_table_load(const int32_t* src, const int32_t* dst, const int64_t* ts,
                                    const int32_t* tag, int64_t nrows, void* stream,
                                    ringo_base** out);
/* Row count of a loaded base table (EINVAL on NULL). */
RINGO_API int ringo_base_table_rows(const ringo_base* b, int64_t* nrows);
/* Releases the table (waits for the device); NULL is a no-op. */
RINGO_API void ringo_base_table_free(ringo_base* b);

/*
 * ringo_select_count -- the number of rows each of preds[0 .. npred)
 * selects, written to the host array counts[npred].  One binary search per
 * (predicate, tag) pair on the device; blocks until done.
 * Errors: EINVAL (NULL b, NULL preds or counts with npred > 0, npred < 0,
 * ntags < 0, NULL tags with ntags > 0), ENOMEM, ECUDA.
 */
RINGO_API int ringo_select_count(const ringo_base* b, const ringo_select* preds, int32_t npred,
                                 void* stream, int64_t* counts);

/*
 * ringo_select_gather -- the rows one predicate selects, written as an edge
 * table into caller-owned device columns d_src[cap], d_dst[cap]: the tags in
 * ascending order, each tag's rows in ts order.  *n receives the row count.
 * Errors: as ringo_select_count; ERANGE if the count exceeds cap (nothing is
 * written, *n still holds the count).
 */
RINGO_API int ringo_select_gather(const ringo_base* b, const ringo_select* pred, int32_t* d_src,
                                  int32_t* d_dst, int64_t cap, int64_t* n, void* stream);

/*
 * ringo_convert_batch -- select and convert npred sub-tables in one batch:
 * graph i is the Section 3.4 conversion of the rows predicate i selects,
 * identical to ringo_table_to_graph of those rows.  All kernels run over
 * every sub-table at once; predicates are taken in order in waves of at most
 * `wave_rows` selected rows (0: the tuned or memory-derived size, see
 * ringo_batch_autotune; a larger single selection forms a wave of its own),
 * which bounds the scratch memory.  Each wave is recorded as one
 * CUDA graph and launched once.  Blocks until done; *out owns the npred
 * graphs until ringo_batch_free.
 * Errors: as ringo_select_count; ERANGE (a selection of 2^31 rows or more),
 * ETIMEOUT (a bounded device wait expired), ENOMEM, ECUDA.  On error *out is
 * NULL and nothing is left allocated.
 */
RINGO_API int ringo_convert_batch(const ringo_base* b, const ringo_select* preds, int32_t npred,
                                  int64_t wave_rows, void* stream, ringo_batch** out);
/*
 * ringo_batch_autotune -- tunes batches of this shape: times
 * ringo_convert_batch with up to four candidate wave sizes (the largest that
 * fits in device memory, then halves, not below 2^24 rows), then, at the
 * fastest size, every radix pass variant (ringo_sort_opts), and records the
 * fastest combination for the GPU and the size class of the mean selection
 * (see ringo_tune_set_cache).  Later ringo_convert_batch calls of that class
 * with wave_rows == 0 use it (the wave capped by what fits in memory then).
 * Without a tuned choice, wave_rows == 0 means the largest wave that fits in
 * 85% of the available device memory, and the default pass variant.
 * Errors: as ringo_convert_batch; ENOMEM if no candidate fits.
 */
RINGO_API int ringo_batch_autotune(const ringo_base* b, const ringo_select* preds, int32_t npred,
                                   void* stream, int64_t* best_wave_rows, double* best_ms);
/* Number of graphs in a batch (= npred). */
RINGO_API int ringo_batch_num_graphs(const ringo_batch* bt, int32_t* n);
/* Sizes and pass counts of graph i, as ringo_graph_get_info gives them for
 * a single graph (EINVAL if i is out of range). */
RINGO_API int ringo_batch_graph_info(const ringo_batch* bt, int32_t i, ringo_graph_info* info);
/* Copies graph i to caller-owned host arrays sized from ringo_batch_graph_info
 * (node_ids[V], offsets[V + 1], neighbours[E]); a NULL array is skipped. */
RINGO_API int ringo_batch_copy_graph_to_host(const ringo_batch* bt, int32_t i,
                                             int32_t* h_node_ids, int64_t* h_out_off,
                                             int32_t* h_out_nbr, int64_t* h_in_off,
                                             int32_t* h_in_nbr);
/* Top-k degrees of graph i (same contract as ringo_graph_degree_topk). */
RINGO_API int ringo_batch_degree_topk(const ringo_batch* bt, int32_t i, int dir, int32_t k,
                                      int32_t* h_ids, int64_t* h_degs, int32_t* n_out);
/* Edge table of graph i (same contract as ringo_graph_to_edge_table; NULL
 * stream: the batch's stream). */
RINGO_API int ringo_batch_graph_to_edge_table(const ringo_batch* bt, int32_t i, int dir,
                                              int32_t* d_src, int32_t* d_dst, int64_t cap,
                                              int64_t* n, void* stream);
/* Releases every graph of the batch; NULL is a no-op. */
RINGO_API void ringo_batch_free(ringo_batch* bt);

/* ------------------------------------------------------------------------
 * Serving: a request loop over a resident base table.
 *
 * A request is select (a predicate as above) + convert (Section 3.4) + the
 * top-k degrees of the graph in both directions.  Worker threads, each with
 * its own CUDA stream, take every request that has arrived when they become
 * free (continuous batching), count the rows each selects, admit requests in
 * arrival order while the device bytes of everything in flight stay within
 * the budget, and run the admitted requests as one wave of the batched
 * pipeline (one CUDA graph).  A request's result is identical to converting
 * its selection alone.  The paper has no serving layer; this is the
 * interactive use of Sections 3.3-3.4 (queries against resident tables).
 * ---------------------------------------------------------------------- */
typedef struct ringo_server ringo_server;
typedef struct ringo_result ringo_result;

typedef struct {
  int32_t workers;         /* concurrent batches (threads and streams); 0: 1, at most 16 */
  int32_t max_batch;       /* requests per batch; 0: 1024 */
  int64_t max_batch_rows;  /* selected rows per batch (a larger single request
                              runs alone); 0: 2^28 */
  int64_t small_rows;      /* requests of at most this many selected rows may
                              also be served by one more worker whose stream
                              has the device's highest priority, so they do
                              not wait out a large wave; 0: 2^21, < 0: none */
} ringo_server_config;

/* submit flag: keep the converted graph with the result (its bytes stay
 * charged to the budget until ringo_result_free). */
#define RINGO_SERVE_KEEP_GRAPH 1

typedef struct {
  int32_t status;          /* RINGO_OK, ENOMEM (larger than the whole budget),
                              ERANGE (2^31 rows or more), ETIMEOUT, ECUDA */
  int32_t batch_requests;  /* requests in the batch that served it */
  int64_t batch_rows;      /* selected rows of that batch */
  int64_t nrows;           /* rows this request selected */
  int64_t num_nodes;       /* V of its graph */
  int64_t num_edges;       /* E of its graph */
  int32_t k_out, k_in;     /* entries in the two top-k lists (min(k, V)) */
  int64_t t_submit_ns;     /* ringo_clock_ns() at submit, admission, completion */
  int64_t t_admit_ns;
  int64_t t_done_ns;
} ringo_result_info;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t batches;                 /* waves run */
  int64_t rows;                    /* selected rows converted */
  int64_t max_concurrent_batches;  /* most batches in flight at once */
  int64_t inflight_bytes;          /* bytes charged to the budget now */
  int64_t max_inflight_bytes;      /* and at most */
  int64_t pending;                 /* submitted, not yet admitted */
} ringo_server_stats;

/* Monotonic clock (nanoseconds) of the result timestamps. */
RINGO_API int64_t ringo_clock_ns(void);

/*
 * ringo_server_create -- starts the workers on the current device.  b stays
 * owned by the caller and must outlive the server.  cfg may be NULL
 * (defaults).  The budget is taken into the library's device memory pool
 * once here (when the device has that much free), so requests do not wait
 * on device memory being mapped; the pool keeps it for later calls.
 * Errors: EINVAL (NULL b or out, budget <= 0, negative workers, max_batch
 * or max_batch_rows), ERANGE (more than 16 workers).
 */
RINGO_API int ringo_server_create(const ringo_base* b, int64_t hbm_budget_bytes,
                                  const ringo_server_config* cfg, ringo_server** out);
/*
 * ringo_server_submit -- queues one request (the predicate's tags are copied)
 * and returns at once with its ticket.  0 <= topk <= 4096 (ERANGE above);
 * flags 0 or RINGO_SERVE_KEEP_GRAPH.  EBUSY once the server is stopping.
 */
RINGO_API int ringo_server_submit(ringo_server* srv, const ringo_select* pred, int32_t topk,
                                  int32_t flags, uint64_t* ticket);
/*
 * ringo_server_wait -- waits up to timeout_us (< 0: no limit) for a ticket's
 * result and hands it to the caller (free with ringo_result_free).  ETIMEOUT
 * if not ready (the ticket stays valid); ENOTFOUND for an unknown or already
 * claimed ticket.  A request's own failure is reported in its info.status.
 */
RINGO_API int ringo_server_wait(ringo_server* srv, uint64_t ticket, int64_t timeout_us,
                                ringo_result** out);
RINGO_API int ringo_server_get_stats(const ringo_server* srv, ringo_server_stats* st);
/* Finishes every submitted request, stops the workers and frees the results
 * nobody claimed.  A request that cannot be admitted because kept graphs the
 * caller still holds fill the budget ends with status EBUSY.  NULL is a
 * no-op. */
RINGO_API void ringo_server_destroy(ringo_server* srv);

RINGO_API int ringo_result_get_info(const ringo_result* r, ringo_result_info* info);
/* Top-k of one direction into caller-owned host arrays of cap entries,
 * degree descending then ID ascending; ERANGE if cap < *n_out. */
RINGO_API int ringo_result_topk(const ringo_result* r, int dir, int32_t* h_ids, int64_t* h_degs,
                                int32_t cap, int32_t* n_out);
/* The kept graph (RINGO_SERVE_KEEP_GRAPH only, else EINVAL), as
 * ringo_batch_copy_graph_to_host. */
RINGO_API int ringo_result_copy_graph_to_host(const ringo_result* r, int32_t* h_node_ids,
                                              int64_t* h_out_off, int32_t* h_out_nbr,
                                              int64_t* h_in_off, int32_t* h_in_nbr);
/* Frees a result (and its kept graph, returning its bytes to the budget). */
RINGO_API void ringo_result_free(ringo_result* r);

/*
 * Kernel timing.  While profiling is on, every kernel the library launches is
 * bracketed by CUDA events on its own stream (kernels recorded into a CUDA
 * graph are timed together, as "batch_wave"), and a few host steps are timed
 * by the wall clock (names starting "host:").  ringo_profile_stop()
 * synchronises the events and returns, per name, the number of launches and
 * their summed time in milliseconds.
 */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
} ringo_kernel_stat;

RINGO_API int ringo_profile_start(void);
RINGO_API int ringo_profile_stop(ringo_kernel_stat* out, int32_t cap, int32_t* n_out);

/*
 * Tuning.  The radix passes have variants that suit different inputs, and
 * batches a wave size; the best choice depends on the GPU and on the data,
 * so it is measured on the caller's own tables and remembered per (GPU
 * name, kind, size class): kind 0 is a single table, 1 a batch, and the size
 * class is floor(log2(rows)) of the table or of the mean selection.  The
 * paper has no counterpart (its conversion runs on CPU threads).
 *   rank_method     0: a warp's lanes with the same digit find each other
 *                      through shared-memory lane masks (default);
 *                   1: through one warp ballot per digit bit (no shared
 *                      atomics: better when many keys share a digit);
 *                   2: through one warp match instruction on the digit
 *   prefetch_waves  0..2: how far ahead, in waves of resident blocks, a
 *                   pass asks L2 for the input of a tile (default 1)
 *   wave_rows       batches only: rows per captured launch (0: automatic)
 *   in_digit_bits   8 or 9: digit width of the in-direction sort passes
 *                   (0 means 8, the default).  With 9-bit digits a table
 *                   with at most 2^27 distinct destinations needs three
 *                   in-direction passes instead of four, each with twice
 *                   the digits.
 *   reserved        0
 * ringo_tune_table -- times the pass variants on this table (device
 *   columns; three conversions each, the first a warm-up: every rank method
 *   and prefetch distance with 8-bit in-direction digits, then every rank
 *   method with 9-bit digits at the best prefetch distance) and records the
 *   fastest for its class; later conversions of that class use it.
 *   *best (and *best_ms, if not NULL) receive the choice.  EINVAL for a NULL
 *   pointer or nrows <= 0; otherwise the errors of ringo_table_to_graph.
 * ringo_tune_lookup -- the recorded choice for (current GPU, kind, class of
 *   rows): *found = 1 and *opts, or *found = 0 and the defaults.
 * ringo_tune_set_cache -- keep the choices in the JSON file at `path`: its
 *   entries are read now (a missing file is created) and it is rewritten
 *   after every new choice, so a later process reuses them.  NULL or "":
 *   memory only.  EINVAL if the file exists and is not a tuning cache.
 * ringo_sort_opts_force -- use these pass options for every conversion
 *   from now on, whatever is recorded (tests and measurements of a
 *   variant); NULL returns to the recorded choices.  EINVAL out of range.
 */
typedef struct {
  int32_t rank_method;
  int32_t prefetch_waves;
  int64_t wave_rows;
  int32_t in_digit_bits;
  int32_t reserved;
} ringo_sort_opts;

RINGO_API int ringo_tune_table(const int32_t* src, const int32_t* dst, int64_t nrows,
                               void* stream, ringo_sort_opts* best, double* best_ms);
RINGO_API int ringo_tune_lookup(int32_t kind, int64_t rows, ringo_sort_opts* opts,
                                int32_t* found);
RINGO_API int ringo_tune_set_cache(const char* path);
RINGO_API int ringo_sort_opts_force(const ringo_sort_opts* opts);

/*
 * Failure-injection hooks for tests of the error paths.  The paper has no
 * counterpart; they make a failure on the host side only, so nothing on the
 * device faults or waits without bound.
 *
 * ringo_test_inject_alloc_failure -- the next `skip` device allocations of
 *   the library succeed and the one after fails (the call that made it
 *   returns RINGO_ENOMEM and frees what it holds); then the hook disarms.
 *   skip < 0 disarms it.  Always RINGO_OK.
 * ringo_test_inject_lookback_timeout -- the next ringo_table_to_graph (or
 *   _host) bounds each of its device waits by spin_limit spins (a spin is a
 *   poll with a short sleep; the default bound is 2^21, about a second) and
 *   its first radix pass never claims tile 0, so the tiles after it wait on
 *   it until the bound: the call returns RINGO_ETIMEOUT and frees what it
 *   holds.  EINVAL unless 1 <= spin_limit <= 2^21.  Taken by the next
 *   conversion on any thread.
 * ringo_test_pool_used -- bytes currently allocated from the library's
 *   device pool on the current device (the pool keeps freed memory cached;
 *   this counts only live allocations, after their stream has reached the
 *   frees).  EINVAL for NULL, ECUDA without a usable device.
 */
RINGO_API int ringo_test_inject_alloc_failure(int32_t skip);
RINGO_API int ringo_test_inject_lookback_timeout(uint32_t spin_limit);
RINGO_API int ringo_test_pool_used(uint64_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* RINGO_H_ */
