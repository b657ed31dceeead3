// Ringo table->graph (and graph->table) ORACLE.  TEST INFRASTRUCTURE ONLY.
//
// This file is the plain, slow, obviously-correct CPU statement of what the
// table->graph conversion computes.  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load it; the product library never links,
// loads or calls it, and it shares no code, header or constant with the CUDA
// path.
//
// Definition followed (paper, Section 3.4 "Conversion of tables to graphs"):
//   * the node set V is the set of unique values found in the source column S
//     and the destination column D;
//   * every row r of the table gives the directed edge (r_S, r_D);
//   * the graph keeps, for every node, a sorted vector of out-neighbours and a
//     sorted vector of in-neighbours (Section 3.2, "Ringo graph
//     representation").
// Readings where the paper is silent (each is listed in the design notes):
//   * duplicate rows collapse to one edge (the neighbour vectors are sorted
//     vectors of a simple directed graph);
//   * self-loops are kept: (u,u) puts u once in out(u) and once in in(u);
//   * node order is ascending signed int32 order, and a node's index is its
//     rank in that order; neighbour entries are node indices;
//   * offsets are int64.
//
// The computation is written as the definition, step by step, with standard
// library primitives only: std::sort + std::unique per direction, and a
// std::map from node ID to node index.
//
// Mutants: when compiled with -DORACLE_MUTANT=k (k>0) one deliberate, plausible
// mistake is planted (see the MUTANT(k) sites).  The pin tests build these
// variants to show that each mistake is caught.  The default build has none.

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <unordered_set>
#include <utility>
#include <vector>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

namespace {

typedef std::pair<int32_t, int32_t> Edge;  // (first, second), signed compare

struct Result {
  std::vector<int32_t> node_ids;
  std::vector<int64_t> out_off, in_off;
  std::vector<int32_t> out_nbr, in_nbr;
};

// Sorted, de-duplicated edge list of one direction.  For the out-direction the
// pair is (src, dst); for the in-direction it is (dst, src).
std::vector<Edge> sorted_unique_edges(const int32_t* first, const int32_t* second,
                                      int64_t n) {
  std::vector<Edge> e;
  e.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    if (MUTANT(4) && first[i] == second[i]) continue;  // drops self-loops
    e.push_back(Edge(first[i], second[i]));
  }
  if (MUTANT(5)) {
    // compares IDs as unsigned: negative IDs sort after positive ones
    std::sort(e.begin(), e.end(), [](const Edge& a, const Edge& b) {
      if ((uint32_t)a.first != (uint32_t)b.first) return (uint32_t)a.first < (uint32_t)b.first;
      return (uint32_t)a.second < (uint32_t)b.second;
    });
  } else {
    std::sort(e.begin(), e.end());
  }
  if (!MUTANT(1)) e.erase(std::unique(e.begin(), e.end()), e.end());
  return e;
}

// CSR of one direction from its sorted unique edge list: offsets indexed by
// node index, neighbours as node indices.
void build_csr(const std::vector<Edge>& e, const std::map<int32_t, int64_t>& index,
               std::vector<int64_t>& off, std::vector<int32_t>& nbr) {
  const size_t V = index.size();
  std::vector<int64_t> count(V, 0);
  for (const Edge& x : e) count[(size_t)index.at(x.first)] += 1;
  off.assign(V + 1, 0);
  for (size_t r = 0; r < V; ++r) off[r + 1] = off[r] + count[r];
  if (MUTANT(3) && V > 0) off[V] -= 1;  // off-by-one in the last offset
  nbr.resize(e.size());
  for (size_t k = 0; k < e.size(); ++k) {
    int64_t r = index.at(e[k].second);
    if (MUTANT(6)) r += 1;  // neighbour index shifted by one
    nbr[k] = (int32_t)r;
  }
}

Result convert(const int32_t* src, const int32_t* dst, int64_t n) {
  Result g;
  // Out-direction: sort (S, D) pairs, drop exact duplicates.
  std::vector<Edge> e_out = sorted_unique_edges(src, dst, n);
  // In-direction: the same edges keyed by destination: sort (D, S) pairs.
  std::vector<Edge> e_in = MUTANT(2) ? sorted_unique_edges(src, dst, n)  // forgets to swap
                                     : sorted_unique_edges(dst, src, n);
  // Node set: unique values of S and D, in ascending order; a std::map gives
  // each ID its index (its rank in key order).
  std::map<int32_t, int64_t> index;
  for (int64_t i = 0; i < n; ++i) {
    index[src[i]] = 0;
    index[dst[i]] = 0;
  }
  int64_t r = 0;
  for (auto& kv : index) kv.second = r++;
  g.node_ids.reserve(index.size());
  for (auto& kv : index) g.node_ids.push_back(kv.first);
  build_csr(e_out, index, g.out_off, g.out_nbr);
  build_csr(e_in, index, g.in_off, g.in_nbr);
  return g;
}

template <class T>
T* export_vec(const std::vector<T>& v) {
  T* p = (T*)std::malloc(sizeof(T) * (v.size() ? v.size() : 1));
  if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

}  // namespace

extern "C" {

// Result arrays are malloc'd here and released by oracle_free.
struct OracleGraph {
  int64_t num_nodes;
  int64_t num_edges;
  int32_t* node_ids;  // [num_nodes]
  int64_t* out_off;   // [num_nodes + 1]
  int32_t* out_nbr;   // [num_edges]
  int64_t* in_off;    // [num_nodes + 1]
  int32_t* in_nbr;    // [num_edges]
};

int oracle_table_to_graph(const int32_t* src, const int32_t* dst, int64_t n,
                          OracleGraph* out) {
  if (!out || n < 0 || (n > 0 && (!src || !dst))) return 1;
  Result g = convert(src, dst, n);
  out->num_nodes = (int64_t)g.node_ids.size();
  out->num_edges = (int64_t)g.out_nbr.size();
  out->node_ids = export_vec(g.node_ids);
  out->out_off = export_vec(g.out_off);
  out->out_nbr = export_vec(g.out_nbr);
  out->in_off = export_vec(g.in_off);
  out->in_nbr = export_vec(g.in_nbr);
  return 0;
}

void oracle_free(OracleGraph* g) {
  if (!g) return;
  std::free(g->node_ids);
  std::free(g->out_off);
  std::free(g->out_nbr);
  std::free(g->in_off);
  std::free(g->in_nbr);
  std::memset(g, 0, sizeof(*g));
}

// Neighbour lists of a few chosen node IDs, straight from the definition, for
// tables too large for oracle_table_to_graph: one scan over the rows collects
// every edge that leaves (out) or enters (in) a chosen node, then each list is
// sorted and de-duplicated.  Lists are given as node IDs (not indices).
//   ids[k]           chosen node IDs (k < nq)
//   out_cnt/in_cnt   [nq] list lengths (output)
//   out_ids/in_ids   concatenated lists, malloc'd here, freed by oracle_free_lists
int oracle_sample_lists(const int32_t* src, const int32_t* dst, int64_t n,
                        const int32_t* ids, int64_t nq, int64_t* out_cnt,
                        int64_t* in_cnt, int32_t** out_ids, int32_t** in_ids,
                        int64_t* present) {
  std::map<int32_t, int64_t> slot;
  for (int64_t k = 0; k < nq; ++k) slot[ids[k]] = k;
  // membership pre-filter (one bit per hash bucket) so that a scan over
  // billions of rows only consults the map for likely matches
  std::vector<uint64_t> filt(1 << 14, 0);
  auto bucket = [](int32_t x) { return (uint32_t)(((uint32_t)x * 2654435761u) >> 12); };
  for (int64_t k = 0; k < nq; ++k) filt[bucket(ids[k]) >> 6] |= 1ull << (bucket(ids[k]) & 63);
  auto maybe = [&](int32_t x) { return (filt[bucket(x) >> 6] >> (bucket(x) & 63)) & 1; };
  std::vector<std::vector<int32_t>> outl(nq), inl(nq);
  std::vector<int64_t> seen(nq, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (maybe(src[i])) {
      auto a = slot.find(src[i]);
      if (a != slot.end()) { outl[a->second].push_back(dst[i]); seen[a->second] = 1; }
    }
    if (maybe(dst[i])) {
      auto b = slot.find(dst[i]);
      if (b != slot.end()) { inl[b->second].push_back(src[i]); seen[b->second] = 1; }
    }
  }
  std::vector<int32_t> oc, ic;
  for (int64_t k = 0; k < nq; ++k) {
    std::sort(outl[k].begin(), outl[k].end());
    outl[k].erase(std::unique(outl[k].begin(), outl[k].end()), outl[k].end());
    std::sort(inl[k].begin(), inl[k].end());
    inl[k].erase(std::unique(inl[k].begin(), inl[k].end()), inl[k].end());
    out_cnt[k] = (int64_t)outl[k].size();
    in_cnt[k] = (int64_t)inl[k].size();
    present[k] = seen[k];
    oc.insert(oc.end(), outl[k].begin(), outl[k].end());
    ic.insert(ic.end(), inl[k].begin(), inl[k].end());
  }
  *out_ids = export_vec(oc);
  *in_ids = export_vec(ic);
  return 0;
}

void oracle_free_lists(int32_t* a, int32_t* b) {
  std::free(a);
  std::free(b);
}

// Number of distinct rows and distinct node IDs of a table, from the
// definition (a hash set per quantity), for size checks on large tables.
int oracle_count_distinct(const int32_t* src, const int32_t* dst, int64_t n,
                          int64_t* num_edges, int64_t* num_nodes) {
  std::unordered_set<uint64_t> rows;
  std::unordered_set<int32_t> nodes;
  rows.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    rows.insert(((uint64_t)(uint32_t)src[i] << 32) | (uint32_t)dst[i]);
    nodes.insert(src[i]);
    nodes.insert(dst[i]);
  }
  *num_edges = (int64_t)rows.size();
  *num_nodes = (int64_t)nodes.size();
  return 0;
}

// Graph -> edge table (paper, Section 3.4 "Conversion of graphs to tables"):
// every node contributes one row per neighbour in one direction's CSR,
// visited node by node, neighbour by neighbour.  Out-CSR rows are
// (node, neighbour); in-CSR rows (swap != 0) are (neighbour, node), so both
// give (src ID, dst ID) columns.
int oracle_graph_to_edge_table(int64_t num_nodes, const int32_t* node_ids, const int64_t* off,
                               const int32_t* nbr, int swap, int32_t* src_out, int32_t* dst_out) {
  int64_t row = 0;
  for (int64_t r = 0; r < num_nodes; ++r) {
    const int64_t end = MUTANT(8) ? off[r + 1] - 1 : off[r + 1];  // drops each last neighbour
    for (int64_t k = off[r]; k < end; ++k) {
      const int32_t node = node_ids[r];
      const int32_t other = node_ids[nbr[k]];
      const bool sw = swap && !MUTANT(7);  // forgets to swap the in-CSR rows back
      src_out[row] = sw ? other : node;
      dst_out[row] = sw ? node : other;
      ++row;
    }
  }
  return 0;
}

// Triangles of an undirected graph given by a symmetric CSR (sorted lists of
// node indices): unordered triples {u, v, w} of distinct nodes with all three
// edges, each counted once as u < v < w: for every u, every neighbour v > u,
// every neighbour w > v of u that is also a neighbour of v.
int oracle_count_triangles(int64_t num_nodes, const int64_t* off, const int32_t* nbr,
                           uint64_t* count) {
  uint64_t c = 0;
  for (int64_t u = 0; u < num_nodes; ++u) {
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      const int64_t v = nbr[i];
      if (v <= u) continue;
      for (int64_t j = off[u]; j < off[u + 1]; ++j) {
        const int64_t w = nbr[j];
        if (MUTANT(9) ? (w == v || w <= u) : (w <= v)) continue;  // mutant: each triangle twice
        if (std::binary_search(nbr + off[v], nbr + off[v + 1], (int32_t)w)) ++c;
      }
    }
  }
  *count = c;
  return 0;
}

}  // extern "C"
