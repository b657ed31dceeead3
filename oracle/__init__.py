"""Ringo table->graph oracle.  TEST INFRASTRUCTURE ONLY.

Plain CPU statement of the conversion defined in the paper's Section 3.4
("Conversion of tables to graphs"): nodes are the unique values of the source
and destination columns, every row is an edge, and each node keeps sorted out-
and in-neighbour vectors (Section 3.2).  The arithmetic lives in
``ringo_oracle.cpp`` (std::sort + std::unique per direction, std::map ID ->
index); this module only compiles it with the host compiler and marshals numpy
arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library neither imports nor links it,
and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ringo_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}


class _OracleGraph(ctypes.Structure):
    _fields_ = [
        ("num_nodes", ctypes.c_int64),
        ("num_edges", ctypes.c_int64),
        ("node_ids", ctypes.POINTER(ctypes.c_int32)),
        ("out_off", ctypes.POINTER(ctypes.c_int64)),
        ("out_nbr", ctypes.POINTER(ctypes.c_int32)),
        ("in_off", ctypes.POINTER(ctypes.c_int64)),
        ("in_nbr", ctypes.POINTER(ctypes.c_int32)),
    ]


def lib_path(mutant: int = 0) -> str:
    name = "libringo_oracle.so" if mutant == 0 else f"libringo_oracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or one planted-mistake variant) with g++."""
    path = lib_path(mutant)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant not in _LIBS:
            lib = ctypes.CDLL(build(mutant))
            lib.oracle_table_to_graph.restype = ctypes.c_int
            lib.oracle_table_to_graph.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_int64, ctypes.POINTER(_OracleGraph)]
            lib.oracle_free.argtypes = [ctypes.POINTER(_OracleGraph)]
            lib.oracle_sample_lists.restype = ctypes.c_int
            lib.oracle_sample_lists.argtypes = [
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)), ctypes.c_void_p]
            lib.oracle_free_lists.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_graph_to_edge_table.restype = ctypes.c_int
            lib.oracle_graph_to_edge_table.argtypes = [
                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_count_triangles.restype = ctypes.c_int
            lib.oracle_count_triangles.argtypes = [ctypes.c_int64, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_count_distinct.restype = ctypes.c_int
            lib.oracle_count_distinct.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_void_p, ctypes.c_void_p]
            _LIBS[mutant] = lib
        return _LIBS[mutant]


def _i32(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a), dtype=np.int32)
    return a


def _take(ptr, n: int, dtype) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def table_to_graph(src, dst, mutant: int = 0) -> dict:
    """Directed graph of an edge table, per the paper's Section 3.4.

    Returns numpy arrays ``node_ids`` (int32, ascending), ``out_off`` /
    ``in_off`` (int64, length V+1) and ``out_nbr`` / ``in_nbr`` (int32 node
    indices, each list strictly increasing).
    """
    s, d = _i32(src), _i32(dst)
    if s.shape != d.shape or s.ndim != 1:
        raise ValueError("src and dst must be 1-D arrays of equal length")
    lib = _lib(mutant)
    g = _OracleGraph()
    rc = lib.oracle_table_to_graph(s.ctypes.data, d.ctypes.data, s.size, ctypes.byref(g))
    if rc != 0:
        raise RuntimeError(f"oracle_table_to_graph failed ({rc})")
    try:
        V, E = int(g.num_nodes), int(g.num_edges)
        return {
            "num_nodes": V,
            "num_edges": E,
            "node_ids": _take(g.node_ids, V, np.int32),
            "out_off": _take(g.out_off, V + 1, np.int64),
            "out_nbr": _take(g.out_nbr, E, np.int32),
            "in_off": _take(g.in_off, V + 1, np.int64),
            "in_nbr": _take(g.in_nbr, E, np.int32),
        }
    finally:
        lib.oracle_free(ctypes.byref(g))


def sample_lists(src, dst, ids) -> tuple[list, list, np.ndarray]:
    """Sorted unique out- and in-neighbour ID lists of the chosen node IDs.

    One scan over all rows (Section 3.4's definition restricted to the chosen
    nodes); usable on tables far too large for :func:`table_to_graph`.
    Returns (out_lists, in_lists, present) with lists of int32 arrays.
    """
    s, d, q = _i32(src), _i32(dst), _i32(ids)
    nq = q.size
    oc = np.zeros(nq, np.int64)
    ic = np.zeros(nq, np.int64)
    pres = np.zeros(nq, np.int64)
    po = ctypes.POINTER(ctypes.c_int32)()
    pi = ctypes.POINTER(ctypes.c_int32)()
    lib = _lib()
    rc = lib.oracle_sample_lists(s.ctypes.data, d.ctypes.data, s.size, q.ctypes.data, nq,
                                 oc.ctypes.data, ic.ctypes.data, ctypes.byref(po),
                                 ctypes.byref(pi), pres.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_sample_lists failed")
    try:
        allo = _take(po, int(oc.sum()), np.int32)
        alli = _take(pi, int(ic.sum()), np.int32)
    finally:
        lib.oracle_free_lists(po, pi)
    oo = np.concatenate([[0], np.cumsum(oc)])
    io = np.concatenate([[0], np.cumsum(ic)])
    outs = [allo[oo[k]:oo[k + 1]] for k in range(nq)]
    ins = [alli[io[k]:io[k + 1]] for k in range(nq)]
    return outs, ins, pres.astype(bool)


def count_distinct(src, dst) -> tuple[int, int]:
    """(number of distinct rows, number of distinct node IDs) of a table."""
    s, d = _i32(src), _i32(dst)
    e = np.zeros(1, np.int64)
    v = np.zeros(1, np.int64)
    _lib().oracle_count_distinct(s.ctypes.data, d.ctypes.data, s.size, e.ctypes.data,
                                 v.ctypes.data)
    return int(e[0]), int(v[0])


def graph_to_edge_table(g: dict, direction: str = "out", mutant: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Edge table of a graph (paper Section 3.4, "Conversion of graphs to
    tables"): (src, dst) ID columns, one row per edge, in the CSR order of
    the chosen direction ("out": by source then destination, "in": by
    destination then source)."""
    V, E = int(g["num_nodes"]), int(g["num_edges"])
    ids = _i32(g["node_ids"])
    off = np.ascontiguousarray(g[f"{direction}_off"], np.int64)
    nbr = _i32(g[f"{direction}_nbr"])
    src = np.zeros(E, np.int32)
    dst = np.zeros(E, np.int32)
    if E:
        rc = _lib(mutant).oracle_graph_to_edge_table(V, ids.ctypes.data, off.ctypes.data,
                                                     nbr.ctypes.data, 1 if direction == "in" else 0,
                                                     src.ctypes.data, dst.ctypes.data)
        if rc != 0:
            raise RuntimeError("oracle_graph_to_edge_table failed")
    return src, dst


def graph_to_node_table(g: dict) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Node table of a graph: node IDs ascending, out-degree, in-degree (the
    lengths of the per-node neighbour vectors)."""
    return (np.asarray(g["node_ids"], np.int32).copy(), np.diff(np.asarray(g["out_off"], np.int64)),
            np.diff(np.asarray(g["in_off"], np.int64)))


def pagerank(g: dict, damping: float = 0.85, iterations: int = 10, drop_dangling: bool = False) -> np.ndarray:
    """PageRank of a built graph (the paper's second workload, Section 4,
    Table "paralg": ten iterations), in fp64, node index order.

    Readings (the paper names the algorithm but not its variant): the
    standard power iteration from the uniform vector,
        PR'(v) = (1 - d) / V + d * ( sum over in-neighbours u of PR(u) / outdeg(u)
                                     + (sum of PR over nodes with no out-edges) / V ),
    with d = damping, a fixed number of iterations and no convergence test.
    ``drop_dangling`` plants a mistake for the pin tests (the mass of nodes
    without out-edges is lost).
    """
    V = int(g["num_nodes"])
    if V == 0:
        return np.zeros(0, np.float64)
    out_off = np.asarray(g["out_off"], np.int64)
    in_off = np.asarray(g["in_off"], np.int64)
    in_nbr = np.asarray(g["in_nbr"], np.int64)
    outdeg = np.diff(out_off)
    indeg = np.diff(in_off)
    row_of_edge = np.repeat(np.arange(V), indeg)  # the node each in-edge enters
    pr = np.full(V, 1.0 / V)
    for _ in range(iterations):
        contrib = np.where(outdeg > 0, pr / np.maximum(outdeg, 1), 0.0)
        dangling = 0.0 if drop_dangling else float(pr[outdeg == 0].sum())
        incoming = np.bincount(row_of_edge, weights=contrib[in_nbr], minlength=V)
        pr = (1.0 - damping) / V + damping * (incoming + dangling / V)
    return pr


def undirected_graph(src, dst) -> dict:
    """The undirected graph of an edge table (the paper's undirected workload,
    Section 4): every row (s, d) is the edge {s, d}, i.e. the directed graph
    of the table with each row also reversed; both CSR directions then hold
    the same symmetric neighbour lists."""
    s, d = _i32(src), _i32(dst)
    return table_to_graph(np.concatenate([s, d]), np.concatenate([d, s]))


def count_triangles(g: dict, mutant: int = 0) -> int:
    """Triangles of the undirected graph in g's (symmetric) out-CSR."""
    off = np.ascontiguousarray(g["out_off"], np.int64)
    nbr = _i32(g["out_nbr"])
    c = np.zeros(1, np.uint64)
    rc = _lib(mutant).oracle_count_triangles(int(g["num_nodes"]), off.ctypes.data, nbr.ctypes.data,
                                             c.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_count_triangles failed")
    return int(c[0])


_OPS = {"<": np.less, "<=": np.less_equal, "==": np.equal, "!=": np.not_equal,
        ">=": np.greater_equal, ">": np.greater}


def table_select(src, dst, col: int, op: str, value: int) -> tuple[np.ndarray, np.ndarray]:
    """Select (Section 3.3; Section 4's select benchmark compares a column with
    a constant): the rows whose column `col` (0: src, 1: dst) compares with
    `value` by `op`, in their order."""
    s, d = _i32(src), _i32(dst)
    keep = _OPS[op](d if col else s, np.int32(value))
    return s[keep], d[keep]


def table_join(src, dst, col: int, keys) -> tuple[np.ndarray, np.ndarray]:
    """Equi-join with a single-column table (Section 4's join benchmark): every
    row whose column `col` value occurs in `keys`, once per occurrence, in row
    order."""
    s, d = _i32(src), _i32(dst)
    key = d if col else s
    uk, cnt = np.unique(_i32(keys), return_counts=True)
    if uk.size == 0 or key.size == 0:
        return s[:0].copy(), d[:0].copy()
    pos = np.minimum(np.searchsorted(uk, key), uk.size - 1)
    mult = np.where(uk[pos] == key, cnt[pos], 0)
    return np.repeat(s, mult), np.repeat(d, mult)
