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
 *   No device or pinned host memory is allocated.  Scratch space is one
 *   fixed __device__ array inside the library (about 41 MB on every GPU that
 *   loads it, held until the process exits), so:
 *   - nrows <= RINGO_NOALLOC_MAX_ROWS, else RINGO_ERANGE;
 *   - calls whose GPU work overlaps (other streams or threads) race on that
 *     array and give wrong results: callers serialise them;
 *   - the first call on each device looks up the array's device address;
 *     make that first call before any stream capture.
 *   src, dst          device columns of nrows int32 IDs (borrowed)
 *   node_ids          device, node_capacity entries       } caller-owned
 *   out_off, in_off   device, node_capacity + 1 entries   } outputs, same
 *   out_nbr, in_nbr   device, edge_capacity entries       } layout as above
 *   edge_capacity     must be >= nrows
 *   node_capacity     must be >= distinct sources + distinct destinations of
 *                     the table (2 * nrows always suffices), else RINGO_ERANGE
 *   num_nodes, num_edges  host outputs: V and E
 * Blocks until the result is complete (two stream synchronisations).
 */
#define RINGO_NOALLOC_MAX_ROWS (1 << 20)
RINGO_API int ringo_table_to_graph_noalloc(const int32_t* src, const int32_t* dst, int64_t nrows,
                                           void* stream, int32_t* node_ids, int64_t* out_off,
                                           int32_t* out_nbr, int64_t* in_off, int32_t* in_nbr,
                                           int64_t node_capacity, int64_t edge_capacity,
                                           int64_t* num_nodes, int64_t* num_edges);

/*
 * Kernel timing.  While profiling is on, every kernel the library launches is
 * bracketed by CUDA events on its own stream.  ringo_profile_stop()
 * synchronises those events and returns, per kernel name, the number of
 * launches and their summed device time.
 */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
} ringo_kernel_stat;

RINGO_API int ringo_profile_start(void);
RINGO_API int ringo_profile_stop(ringo_kernel_stat* out, int32_t cap, int32_t* n_out);

#ifdef __cplusplus
}
#endif

#endif /* RINGO_H_ */
