"""Pins for the table->graph conversion: checks that do not trust any
implementation under test.

* ``load_golden``: hand-worked tables (tests/golden/, each citing the paper).
* ``brute_force``: the definition computed a different way, through a dense
  boolean adjacency matrix over the sorted node set (pure Python; tiny inputs).
* ``check_invariants``: properties every correct result has (paper Section 3.4
  and Section 3.2): degree sums equal the number of distinct rows, v in out(u)
  iff u in in(v), every list strictly increasing, node IDs strictly increasing,
  every node has an edge, and the node set is exactly the set of IDs in the
  two columns.
* ``check_special_cases``: closed forms for structured tables.

Every function raises AssertionError on a mismatch.  Each takes a
``convert(src, dst) -> dict`` callable so the same pins can be aimed at the
oracle or at a planted-mistake variant of it.
"""
from __future__ import annotations

import os
import itertools

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ARRAYS = ("node_ids", "out_off", "out_nbr", "in_off", "in_nbr")


def load_golden(path: str) -> dict:
    out: dict = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(":")
            key, toks = key.strip(), val.split()
            if key == "rows":
                pairs = [tuple(int(x) for x in t.split(",")) for t in toks]
                out["src"] = np.array([p[0] for p in pairs], np.int32)
                out["dst"] = np.array([p[1] for p in pairs], np.int32)
            elif key in ("num_nodes", "num_edges"):
                out[key] = int(toks[0])
            else:
                dt = np.int64 if key.endswith("_off") else np.int32
                out[key] = np.array([int(x) for x in toks], dt)
    return out


def golden_files() -> list[str]:
    return sorted(os.path.join(GOLDEN_DIR, f) for f in os.listdir(GOLDEN_DIR)
                  if f.endswith(".txt"))


def assert_same_graph(got: dict, want: dict, what: str = "") -> None:
    assert int(got["num_nodes"]) == int(want["num_nodes"]), \
        f"{what}: num_nodes {got['num_nodes']} != {want['num_nodes']}"
    assert int(got["num_edges"]) == int(want["num_edges"]), \
        f"{what}: num_edges {got['num_edges']} != {want['num_edges']}"
    for k in ARRAYS:
        a = np.asarray(got[k]).astype(np.int64)
        b = np.asarray(want[k]).astype(np.int64)
        assert a.shape == b.shape, f"{what}: {k} shape {a.shape} != {b.shape}"
        if not np.array_equal(a, b):
            bad = int(np.flatnonzero(a != b)[0])
            raise AssertionError(f"{what}: {k} differs first at {bad}: {a[bad]} != {b[bad]}")


def brute_force(src, dst) -> dict:
    """Definition via a dense adjacency matrix (pure Python, tiny inputs).

    Node set = sorted set of all values in both columns; A[i][j] is True when
    some row goes from node i to node j.  Row i of A read left to right is
    node i's sorted out-list; column j read top to bottom is its in-list.
    """
    s = [int(x) for x in src]
    d = [int(x) for x in dst]
    ids = sorted(set(s) | set(d))
    pos = {v: i for i, v in enumerate(ids)}
    V = len(ids)
    A = [[False] * V for _ in range(V)]
    for a, b in zip(s, d):
        A[pos[a]][pos[b]] = True
    out_off, out_nbr, in_off, in_nbr = [0], [], [0], []
    for i in range(V):
        for j in range(V):
            if A[i][j]:
                out_nbr.append(j)
        out_off.append(len(out_nbr))
    for j in range(V):
        for i in range(V):
            if A[i][j]:
                in_nbr.append(i)
        in_off.append(len(in_nbr))
    return {
        "num_nodes": V, "num_edges": len(out_nbr),
        "node_ids": np.array(ids, np.int32), "out_off": np.array(out_off, np.int64),
        "out_nbr": np.array(out_nbr, np.int32), "in_off": np.array(in_off, np.int64),
        "in_nbr": np.array(in_nbr, np.int32),
    }


def _edges_of(off, nbr) -> np.ndarray:
    """(owner index, neighbour index) for every CSR entry."""
    off = np.asarray(off, np.int64)
    deg = np.diff(off)
    owner = np.repeat(np.arange(deg.size, dtype=np.int64), deg)
    return np.stack([owner, np.asarray(nbr, np.int64)], axis=1)


def check_invariants(g: dict, src, dst) -> None:
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    ids = np.asarray(g["node_ids"], np.int64)
    V, E = int(g["num_nodes"]), int(g["num_edges"])
    assert ids.size == V
    # node set is exactly the set of values of the two columns
    want_ids = np.unique(np.concatenate([src, dst]))
    assert np.array_equal(ids, want_ids), "node set is not the unique values of S and D"
    for dirn in ("out", "in"):
        off = np.asarray(g[f"{dirn}_off"], np.int64)
        nbr = np.asarray(g[f"{dirn}_nbr"], np.int64)
        assert off.size == V + 1 and off[0] == 0 and off[-1] == E, f"{dirn}_off ends"
        assert np.all(np.diff(off) >= 0), f"{dirn}_off not monotone"
        assert nbr.size == E
        if E:
            assert nbr.min() >= 0 and nbr.max() < V, f"{dirn}_nbr out of range"
            # strictly increasing inside every list
            inside = np.ones(E, bool)
            inside[off[:-1][np.diff(off) > 0]] = False
            step = np.diff(nbr)
            assert np.all(step[inside[1:]] > 0), f"{dirn} list not strictly increasing"
    # E equals the number of distinct rows
    keys = (src << 32) ^ (dst & 0xFFFFFFFF)
    assert E == np.unique(keys).size, "E != number of distinct rows"
    # v in out(u) iff u in in(v): the out edge set equals the transposed in set
    eo = _edges_of(g["out_off"], g["out_nbr"])
    ei = _edges_of(g["in_off"], g["in_nbr"])[:, ::-1]
    ko = eo[:, 0] * max(V, 1) + eo[:, 1]
    ki = ei[:, 0] * max(V, 1) + ei[:, 1]
    assert np.array_equal(np.sort(ko), np.sort(ki)), "out and in edge sets disagree"
    # each edge is a row of the table, mapped through node_ids
    if E:
        rows = np.unique(keys)
        ek = (ids[eo[:, 0]] << 32) ^ (ids[eo[:, 1]] & 0xFFFFFFFF)
        assert np.array_equal(np.sort(ek), rows), "edge set is not the set of rows"
    # every node touches an edge
    deg = np.diff(np.asarray(g["out_off"], np.int64)) + np.diff(np.asarray(g["in_off"], np.int64))
    assert V == 0 or deg.min() >= 1, "a node without edges"


def check_golden(convert) -> None:
    for path in golden_files():
        want = load_golden(path)
        got = convert(want["src"], want["dst"])
        assert_same_graph(got, want, os.path.basename(path))


def exhaustive_tables(alphabet=(-1, 0, 1, 2), max_rows: int = 4):
    rows = [(a, b) for a in alphabet for b in alphabet]
    for k in range(max_rows + 1):
        for combo in itertools.product(rows, repeat=k):
            yield (np.array([r[0] for r in combo], np.int32),
                   np.array([r[1] for r in combo], np.int32))


def check_brute_force_exhaustive(convert, alphabet=(-1, 0, 1, 2), max_rows: int = 4) -> int:
    n = 0
    for s, d in exhaustive_tables(alphabet, max_rows):
        assert_same_graph(convert(s, d), brute_force(s, d), f"table {list(zip(s, d))}")
        n += 1
    return n


def check_brute_force_random(convert, trials: int = 300, seed: int = 7) -> None:
    rng = np.random.default_rng(seed)
    pool = np.array([-2**31, -2**31 + 1, -5, -1, 0, 1, 3, 2**31 - 2, 2**31 - 1], np.int64)
    for t in range(trials):
        n = int(rng.integers(0, 12))
        s = pool[rng.integers(0, pool.size, n)].astype(np.int32)
        d = pool[rng.integers(0, pool.size, n)].astype(np.int32)
        assert_same_graph(convert(s, d), brute_force(s, d), f"random table {t}")


def check_special_cases(convert) -> None:
    rng = np.random.default_rng(11)
    # distinct sources, no duplicates: out-CSR is a permutation, E = N, every
    # source has out-degree exactly 1
    n = 500
    s = rng.choice(np.arange(-10**6, 10**6), size=n, replace=False).astype(np.int32)
    d = rng.integers(-10**6, 10**6, n).astype(np.int32)
    g = convert(s, d)
    assert g["num_edges"] == n
    ids = np.asarray(g["node_ids"], np.int64)
    r = np.searchsorted(ids, s)
    outdeg = np.diff(np.asarray(g["out_off"], np.int64))
    assert np.all(outdeg[r] == 1)
    assert np.array_equal(ids[np.asarray(g["out_nbr"])[np.asarray(g["out_off"])[r]]], d)
    # a directed path 0->1->...->m-1 with scrambled row order: node i has
    # out-list [i+1] and in-list [i-1]
    m = 64
    perm = rng.permutation(m - 1)
    s = np.arange(m - 1, dtype=np.int32)[perm]
    d = (np.arange(m - 1, dtype=np.int32) + 1)[perm]
    g = convert(s, d)
    assert np.array_equal(np.asarray(g["out_off"]), np.r_[np.arange(m), m - 1])
    assert np.array_equal(np.asarray(g["out_nbr"]), np.arange(1, m))
    assert np.array_equal(np.asarray(g["in_off"]), np.r_[0, np.arange(m)])
    assert np.array_equal(np.asarray(g["in_nbr"]), np.arange(0, m - 1))
    # complete digraph with loops on k nodes: every list is 0..k-1
    k = 9
    a, b = np.meshgrid(np.arange(k) * 7 - 20, np.arange(k) * 7 - 20, indexing="ij")
    g = convert(a.ravel().astype(np.int32)[::-1], b.ravel().astype(np.int32)[::-1])
    assert g["num_edges"] == k * k
    assert np.array_equal(np.asarray(g["out_nbr"]), np.tile(np.arange(k), k))
    assert np.array_equal(np.asarray(g["in_nbr"]), np.tile(np.arange(k), k))


def check_row_order_and_duplicates(convert, src, dst, seed: int = 3) -> None:
    """Result is independent of row order and of adding duplicate rows."""
    base = convert(src, dst)
    rng = np.random.default_rng(seed)
    p = rng.permutation(len(src))
    assert_same_graph(convert(np.asarray(src)[p], np.asarray(dst)[p]), base, "shuffled")
    if len(src):
        extra = rng.integers(0, len(src), max(1, len(src) // 10))
        s2 = np.concatenate([src, np.asarray(src)[extra]])
        d2 = np.concatenate([dst, np.asarray(dst)[extra]])
        assert_same_graph(convert(s2, d2), base, "with duplicates")


# ------------------------------------------------------------ graph -> table
def expected_tables(src, dst) -> dict:
    """Section 3.4, "Conversion of graphs to tables", on the graph of a table:
    one edge-table row per distinct row of the table (set semantics), in
    (src, dst) order for the out-CSR and (dst, src) order for the in-CSR;
    one node-table row per distinct ID, with the number of distinct rows that
    leave and that enter it.  Plain Python sets and sorts."""
    rows = sorted(set(zip((int(x) for x in src), (int(x) for x in dst))))
    rows_in = sorted(rows, key=lambda r: (r[1], r[0]))
    ids = sorted(set(int(x) for x in src) | set(int(x) for x in dst))
    outdeg = {i: 0 for i in ids}
    indeg = {i: 0 for i in ids}
    for a, b in rows:
        outdeg[a] += 1
        indeg[b] += 1
    col = lambda xs: np.array(xs, dtype=np.int32)
    return {"out_src": col([r[0] for r in rows]), "out_dst": col([r[1] for r in rows]),
            "in_src": col([r[0] for r in rows_in]), "in_dst": col([r[1] for r in rows_in]),
            "ids": col(ids), "outdeg": np.array([outdeg[i] for i in ids], np.int64),
            "indeg": np.array([indeg[i] for i in ids], np.int64)}


def assert_same_tables(got: dict, want: dict, what: str = "") -> None:
    for k in ("out_src", "out_dst", "in_src", "in_dst", "ids", "outdeg", "indeg"):
        g, w = np.asarray(got[k]), np.asarray(want[k])
        assert g.shape == w.shape and np.array_equal(g, w), f"{what}: {k} differs"


def check_graph_to_table(tables, max_rows: int = 3, trials: int = 100, seed: int = 11) -> None:
    """`tables(src, dst)` returns the edge tables (both directions) and the
    node table of the graph of (src, dst); checked on the golden tables, every
    table of up to max_rows rows over {-1, 0, 1, 2}, and random tables over
    extreme IDs."""
    for path in golden_files():
        t = load_golden(path)
        assert_same_tables(tables(t["src"], t["dst"]), expected_tables(t["src"], t["dst"]),
                           os.path.basename(path))
    for s, d in exhaustive_tables(max_rows=max_rows):
        assert_same_tables(tables(s, d), expected_tables(s, d), f"{s.tolist()} {d.tolist()}")
    rng = np.random.default_rng(seed)
    pool = np.array([-2**31, -2**31 + 1, -7, -1, 0, 1, 5, 2**31 - 2, 2**31 - 1], np.int32)
    for _ in range(trials):
        n = int(rng.integers(0, 40))
        s = pool[rng.integers(0, pool.size, n)]
        d = pool[rng.integers(0, pool.size, n)]
        assert_same_tables(tables(s, d), expected_tables(s, d), "random")
