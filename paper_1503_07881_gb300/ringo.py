"""Python binding of libringo (the C ABI in include/ringo.h).

Argument marshalling only: every step of the conversion runs in the CUDA
library.  PyTorch is used for device memory and streams: columns are passed
as ``tensor.data_ptr()``, the stream as ``torch.cuda.current_stream()``.

If the compiled library is missing this module raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

RINGO_OK, RINGO_EINVAL, RINGO_ENOMEM, RINGO_ECUDA = 0, 1, 2, 3
RINGO_ETIMEOUT, RINGO_ENOTFOUND, RINGO_EBUSY, RINGO_ERANGE = 4, 5, 6, 7
RINGO_OUT, RINGO_IN = 0, 1

_lib = None


class RingoError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_name(status)}) {detail}".strip())


def _status_name(s: int) -> str:
    return {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTFOUND",
            6: "EBUSY", 7: "ERANGE"}.get(s, "unknown")


class GraphInfo(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("num_nodes", ctypes.c_int64),
                ("num_edges", ctypes.c_int64), ("num_src_nodes", ctypes.c_int64),
                ("num_dst_nodes", ctypes.c_int64), ("out_sort_passes", ctypes.c_int32),
                ("in_sort_passes", ctypes.c_int32)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


# every symbol include/ringo.h declares, with its ctypes signature
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "ringo_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ringo_last_error": (ctypes.c_char_p, []),
    "ringo_version": (ctypes.c_char_p, []),
    "ringo_table_to_graph": (ctypes.c_int, [_P, _P, _I64, _P, _PP]),
    "ringo_table_to_graph_host": (ctypes.c_int, [_P, _P, _I64, _P, _PP]),
    "ringo_graph_num_nodes": (ctypes.c_int, [_P, _P]),
    "ringo_graph_num_edges": (ctypes.c_int, [_P, _P]),
    "ringo_graph_get_info": (ctypes.c_int, [_P, ctypes.POINTER(GraphInfo)]),
    "ringo_graph_node_ids": (ctypes.c_int, [_P, _PP]),
    "ringo_graph_csr": (ctypes.c_int, [_P, ctypes.c_int, _PP, _PP]),
    "ringo_graph_degree": (ctypes.c_int, [_P, ctypes.c_int, _I32, _P]),
    "ringo_graph_degrees": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _P, _P]),
    "ringo_graph_degree_topk": (ctypes.c_int, [_P, ctypes.c_int, _I32, _P, _P, _P]),
    "ringo_graph_copy_to_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "ringo_graph_free": (None, [_P]),
    "ringo_table_to_graph_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _I64,
                                                    _I64, _P, _P]),
    "ringo_base_table_load": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _PP]),
    "ringo_base_table_rows": (ctypes.c_int, [_P, _P]),
    "ringo_base_table_free": (None, [_P]),
    "ringo_select_count": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "ringo_select_gather": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "ringo_convert_batch": (ctypes.c_int, [_P, _P, _I32, _I64, _P, _PP]),
    "ringo_batch_autotune": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "ringo_batch_num_graphs": (ctypes.c_int, [_P, _P]),
    "ringo_batch_graph_info": (ctypes.c_int, [_P, _I32, ctypes.POINTER(GraphInfo)]),
    "ringo_batch_copy_graph_to_host": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    "ringo_batch_degree_topk": (ctypes.c_int, [_P, _I32, ctypes.c_int, _I32, _P, _P, _P]),
    "ringo_batch_free": (None, [_P]),
    "ringo_clock_ns": (ctypes.c_int64, []),
    "ringo_server_create": (ctypes.c_int, [_P, _I64, _P, _PP]),
    "ringo_server_submit": (ctypes.c_int, [_P, _P, _I32, _I32, ctypes.POINTER(ctypes.c_uint64)]),
    "ringo_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _I64, _PP]),
    "ringo_server_get_stats": (ctypes.c_int, [_P, _P]),
    "ringo_server_destroy": (None, [_P]),
    "ringo_result_get_info": (ctypes.c_int, [_P, _P]),
    "ringo_result_topk": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _I32, _P]),
    "ringo_result_copy_graph_to_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "ringo_result_free": (None, [_P]),
    "ringo_graph_to_edge_table": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _I64, _P, _P]),
    "ringo_graph_to_node_table": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "ringo_batch_graph_to_edge_table": (ctypes.c_int, [_P, _I32, ctypes.c_int, _P, _P, _I64, _P,
                                                       _P]),
    "ringo_graph_pagerank": (ctypes.c_int, [_P, ctypes.c_double, _I32, _P, _P]),
    "ringo_table_to_undirected_graph": (ctypes.c_int, [_P, _P, _I64, _P, _PP]),
    "ringo_table_to_graph_host_io": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _I64,
                                                    _I64, _P, _P]),
    "ringo_graph_count_triangles": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "ringo_table_select": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, ctypes.c_int, _I32, _P, _P]),
    "ringo_table_join": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I64, _P, _P, _I64, _P,
                                        _P]),
    "ringo_tune_table": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "ringo_tune_lookup": (ctypes.c_int, [_I32, _I64, _P, _P]),
    "ringo_tune_set_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "ringo_sort_opts_force": (ctypes.c_int, [_P]),
    "ringo_test_inject_alloc_failure": (ctypes.c_int, [_I32]),
    "ringo_test_inject_lookback_timeout": (ctypes.c_int, [ctypes.c_uint32]),
    "ringo_test_pool_used": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "ringo_profile_start": (ctypes.c_int, []),
    "ringo_profile_stop": (ctypes.c_int, [ctypes.POINTER(KernelStat), _I32, _P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libringo.so (building it in-tree with nvcc if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libringo.so not built ({path}); run build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str) -> None:
    if rc != RINGO_OK:
        detail = load().ringo_last_error().decode(errors="replace")
        raise RingoError(rc, where, detail)


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class _DevArray:
    """Borrowed device array exposed through __cuda_array_interface__; keeps
    its graph alive while a tensor views it."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
            "strides": None, "stream": None,
        }


def _view(ptr, n: int, dtype: torch.dtype, owner) -> torch.Tensor:
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    typestr = {torch.int32: "<i4", torch.int64: "<i8"}[dtype]
    return torch.as_tensor(_DevArray(int(ptr), n, typestr, owner), device="cuda")


class Graph:
    """Owner of a ``ringo_graph*`` handle."""

    def __init__(self, handle: int, stream_ptr: int):
        self._h = ctypes.c_void_p(handle)
        self._stream_ptr = stream_ptr

    def __del__(self):
        self.free()

    def free(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            load().ringo_graph_free(self._h)
            self._h = ctypes.c_void_p(0)

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h.value:
            raise RuntimeError("graph already freed")
        return self._h

    def info(self) -> dict:
        gi = GraphInfo()
        _check(load().ringo_graph_get_info(self.handle, ctypes.byref(gi)), "ringo_graph_get_info")
        return {f: getattr(gi, f) for f, _ in GraphInfo._fields_}

    @property
    def num_nodes(self) -> int:
        v = ctypes.c_int64()
        _check(load().ringo_graph_num_nodes(self.handle, ctypes.byref(v)), "ringo_graph_num_nodes")
        return v.value

    @property
    def num_edges(self) -> int:
        e = ctypes.c_int64()
        _check(load().ringo_graph_num_edges(self.handle, ctypes.byref(e)), "ringo_graph_num_edges")
        return e.value

    def node_ids(self) -> torch.Tensor:
        p = ctypes.c_void_p()
        _check(load().ringo_graph_node_ids(self.handle, ctypes.byref(p)), "ringo_graph_node_ids")
        return _view(p.value, self.num_nodes, torch.int32, self)

    def csr(self, direction: int = RINGO_OUT) -> tuple[torch.Tensor, torch.Tensor]:
        po, pn = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().ringo_graph_csr(self.handle, direction, ctypes.byref(po), ctypes.byref(pn)),
               "ringo_graph_csr")
        return (_view(po.value, self.num_nodes + 1, torch.int64, self),
                _view(pn.value, self.num_edges, torch.int32, self))

    def degree(self, direction: int, node_id: int) -> int:
        d = ctypes.c_int64()
        _check(load().ringo_graph_degree(self.handle, direction, int(node_id), ctypes.byref(d)),
               "ringo_graph_degree")
        return d.value

    def degrees(self, direction: int, ids: torch.Tensor, stream=None) -> torch.Tensor:
        ids = ids.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(ids.numel(), dtype=torch.int64, device="cuda")
        _check(load().ringo_graph_degrees(self.handle, direction, ids.data_ptr(), ids.numel(),
                                          out.data_ptr(), _stream_ptr(stream)),
               "ringo_graph_degrees")
        return out

    def degree_topk(self, direction: int, k: int) -> tuple[np.ndarray, np.ndarray]:
        ids = np.zeros(max(k, 1), np.int32)
        degs = np.zeros(max(k, 1), np.int64)
        n = ctypes.c_int32()
        _check(load().ringo_graph_degree_topk(self.handle, direction, int(k), ids.ctypes.data,
                                              degs.ctypes.data, ctypes.byref(n)),
               "ringo_graph_degree_topk")
        return ids[:n.value].copy(), degs[:n.value].copy()

    def to_edge_table(self, direction: int = RINGO_OUT, out=None,
                      stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """Section 3.4 graph -> table: (src, dst) ID columns, one row per edge,
        in the CSR order of `direction`.  `out` may give two int32 CUDA tensors
        of at least E entries."""
        E = self.num_edges
        if out is None:
            out = (torch.empty(max(E, 1), dtype=torch.int32, device="cuda"),
                   torch.empty(max(E, 1), dtype=torch.int32, device="cuda"))
        src, dst = out
        n = ctypes.c_int64()
        _check(load().ringo_graph_to_edge_table(self.handle, direction, src.data_ptr(),
                                                dst.data_ptr(), min(src.numel(), dst.numel()),
                                                ctypes.byref(n), _stream_ptr(stream)),
               "ringo_graph_to_edge_table")
        return src[:n.value], dst[:n.value]

    def pagerank(self, damping: float = 0.85, iterations: int = 10, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
        """PageRank (fp64, node index order) as a CUDA tensor."""
        V = self.num_nodes
        if out is None:
            out = torch.empty(max(V, 1), dtype=torch.float64, device="cuda")
        _check(load().ringo_graph_pagerank(self.handle, float(damping), int(iterations),
                                           out.data_ptr(), _stream_ptr(stream)),
               "ringo_graph_pagerank")
        return out[:V]

    def count_triangles(self, stream=None) -> int:
        """Triangles of the undirected graph in the out-CSR (see
        ringo_table_to_undirected_graph)."""
        c = ctypes.c_uint64()
        _check(load().ringo_graph_count_triangles(self.handle, _stream_ptr(stream), ctypes.byref(c)),
               "ringo_graph_count_triangles")
        return c.value

    def to_node_table(self, stream=None) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
        """(node IDs ascending, out-degree, in-degree) as CUDA tensors."""
        V = self.num_nodes
        ids = torch.empty(max(V, 1), dtype=torch.int32, device="cuda")
        od = torch.empty(max(V, 1), dtype=torch.int64, device="cuda")
        idg = torch.empty(max(V, 1), dtype=torch.int64, device="cuda")
        n = ctypes.c_int64()
        _check(load().ringo_graph_to_node_table(self.handle, ids.data_ptr(), od.data_ptr(),
                                                idg.data_ptr(), V, ctypes.byref(n),
                                                _stream_ptr(stream)),
               "ringo_graph_to_node_table")
        return ids[:V], od[:V], idg[:V]

    def copy_to_host(self, out: dict | None = None) -> dict:
        """All five arrays into host memory (numpy, or caller-given buffers)."""
        V, E = self.num_nodes, self.num_edges
        if out is None:
            out = {"node_ids": np.empty(V, np.int32), "out_off": np.empty(V + 1, np.int64),
                   "out_nbr": np.empty(E, np.int32), "in_off": np.empty(V + 1, np.int64),
                   "in_nbr": np.empty(E, np.int32)}

        def ptr(a):
            if isinstance(a, torch.Tensor):
                return a.data_ptr()
            return a.ctypes.data

        _check(load().ringo_graph_copy_to_host(
            self.handle, ptr(out["node_ids"]), ptr(out["out_off"]), ptr(out["out_nbr"]),
            ptr(out["in_off"]), ptr(out["in_nbr"])), "ringo_graph_copy_to_host")
        res = dict(out)
        res["num_nodes"], res["num_edges"] = V, E
        return res


def _col_ptr(t: torch.Tensor, name: str) -> int:
    if t.dtype != torch.int32 or t.dim() != 1:
        raise ValueError(f"{name} must be a 1-D int32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def ringo_table_to_graph(src: torch.Tensor, dst: torch.Tensor, stream=None) -> Graph:
    """Section 3.4 conversion of device columns (int32 CUDA tensors)."""
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    if src.numel() and (not src.is_cuda or not dst.is_cuda):
        raise ValueError("columns must be CUDA tensors; use ringo_table_to_graph_host")
    lib = load()
    sp = _stream_ptr(stream)
    h = ctypes.c_void_p()
    _check(lib.ringo_table_to_graph(_col_ptr(src, "src") if src.numel() else None,
                                    _col_ptr(dst, "dst") if dst.numel() else None,
                                    src.numel(), sp, ctypes.byref(h)), "ringo_table_to_graph")
    return Graph(h.value, sp)


def ringo_table_to_undirected_graph(src: torch.Tensor, dst: torch.Tensor, stream=None) -> Graph:
    """Undirected graph of device columns: each row is the edge {src, dst}."""
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    if src.numel() and (not src.is_cuda or not dst.is_cuda):
        raise ValueError("columns must be CUDA tensors")
    sp = _stream_ptr(stream)
    h = ctypes.c_void_p()
    _check(load().ringo_table_to_undirected_graph(_col_ptr(src, "src") if src.numel() else None,
                                                  _col_ptr(dst, "dst") if dst.numel() else None,
                                                  src.numel(), sp, ctypes.byref(h)),
           "ringo_table_to_undirected_graph")
    return Graph(h.value, sp)


def ringo_table_to_graph_host(src, dst, stream=None) -> Graph:
    """The same conversion from host columns (numpy arrays or CPU tensors;
    pinned CPU tensors copy fastest)."""
    def hptr(a):
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.int32 or not a.is_contiguous():
                raise ValueError("host column must be a contiguous CPU int32 tensor")
            return a.data_ptr(), a.numel(), a
        a = np.ascontiguousarray(a, dtype=np.int32)
        return a.ctypes.data, a.size, a

    ps, ns, keep_s = hptr(src)
    pd, nd, keep_d = hptr(dst)
    if ns != nd:
        raise ValueError("src and dst differ in length")
    lib = load()
    sp = _stream_ptr(stream)
    h = ctypes.c_void_p()
    _check(lib.ringo_table_to_graph_host(ps if ns else None, pd if nd else None, ns, sp,
                                         ctypes.byref(h)), "ringo_table_to_graph_host")
    del keep_s, keep_d
    return Graph(h.value, sp)


def ringo_table_to_graph_host_io(src, dst, out: dict | None = None, stream=None) -> dict:
    """Host columns in, host arrays out, in one call (the out-CSR comes
    back while the in-CSR is built).  ``out`` may hold caller-owned CPU
    tensors (pinned ones copy fastest): int32 ``node_ids`` / ``out_nbr`` /
    ``in_nbr`` and int64 ``out_off`` / ``in_off`` with room for 2 * nrows
    nodes and nrows edges; without it, pinned tensors of that size are made.
    Returns a dict of views of the five arrays plus num_nodes / num_edges."""
    def hptr(a):
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.int32 or not a.is_contiguous():
                raise ValueError("host column must be a contiguous CPU int32 tensor")
            return a.data_ptr(), a.numel(), a
        a = np.ascontiguousarray(a, dtype=np.int32)
        return a.ctypes.data, a.size, a

    ps, ns, keep_s = hptr(src)
    pd, nd, keep_d = hptr(dst)
    if ns != nd:
        raise ValueError("src and dst differ in length")
    if out is None:
        pin = torch.cuda.is_available()
        out = {"node_ids": torch.empty(2 * ns, dtype=torch.int32, pin_memory=pin),
               "out_off": torch.empty(2 * ns + 1, dtype=torch.int64, pin_memory=pin),
               "out_nbr": torch.empty(max(ns, 1), dtype=torch.int32, pin_memory=pin),
               "in_off": torch.empty(2 * ns + 1, dtype=torch.int64, pin_memory=pin),
               "in_nbr": torch.empty(max(ns, 1), dtype=torch.int32, pin_memory=pin)}
    want = {"node_ids": torch.int32, "out_off": torch.int64, "out_nbr": torch.int32,
            "in_off": torch.int64, "in_nbr": torch.int32}
    for name, dtype in want.items():
        t = out.get(name)
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"out[{name!r}] must be a contiguous CPU {dtype} tensor")
    node_cap = out["node_ids"].numel()
    if min(out["out_off"].numel(), out["in_off"].numel()) < node_cap + 1:
        raise ValueError("out_off and in_off need node_ids.numel() + 1 entries")
    v, e = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ringo_table_to_graph_host_io(
        ps if ns else None, pd if nd else None, ns, _stream_ptr(stream),
        out["node_ids"].data_ptr(), out["out_off"].data_ptr(), out["out_nbr"].data_ptr(),
        out["in_off"].data_ptr(), out["in_nbr"].data_ptr(), node_cap,
        min(out["out_nbr"].numel(), out["in_nbr"].numel()), ctypes.byref(v), ctypes.byref(e)),
        "ringo_table_to_graph_host_io")
    del keep_s, keep_d
    V, E = v.value, e.value
    return {"num_nodes": V, "num_edges": E, "node_ids": out["node_ids"][:V],
            "out_off": out["out_off"][:V + 1], "out_nbr": out["out_nbr"][:E],
            "in_off": out["in_off"][:V + 1], "in_nbr": out["in_nbr"][:E]}


def ringo_profile_start() -> None:
    _check(load().ringo_profile_start(), "ringo_profile_start")


def ringo_profile_stop() -> list[dict]:
    cap = 64
    arr = (KernelStat * cap)()
    n = ctypes.c_int32()
    _check(load().ringo_profile_stop(arr, cap, ctypes.byref(n)), "ringo_profile_stop")
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches,
             "total_ms": arr[i].total_ms} for i in range(min(n.value, cap))]


class SortOpts(ctypes.Structure):
    _fields_ = [("rank_method", ctypes.c_int32), ("prefetch_waves", ctypes.c_int32),
                ("wave_rows", ctypes.c_int64), ("in_digit_bits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _opts_dict(o: SortOpts) -> dict:
    return {"rank_method": o.rank_method, "prefetch_waves": o.prefetch_waves,
            "wave_rows": o.wave_rows, "in_digit_bits": o.in_digit_bits}


def ringo_tune_table(src: torch.Tensor, dst: torch.Tensor, stream=None) -> tuple[dict, float]:
    """Times every radix pass variant on this table and records the fastest
    for its size class; returns (options, ms)."""
    o, ms = SortOpts(), ctypes.c_double()
    _check(load().ringo_tune_table(_col_ptr(src, "src"), _col_ptr(dst, "dst"), src.numel(),
                                   _stream_ptr(stream), ctypes.byref(o), ctypes.byref(ms)),
           "ringo_tune_table")
    return _opts_dict(o), ms.value


def ringo_tune_lookup(kind: int, rows: int) -> tuple[bool, dict]:
    """The recorded choice for (this GPU, kind 0 table / 1 batch, class of rows)."""
    o, found = SortOpts(), ctypes.c_int32()
    _check(load().ringo_tune_lookup(int(kind), int(rows), ctypes.byref(o), ctypes.byref(found)),
           "ringo_tune_lookup")
    return bool(found.value), _opts_dict(o)


def ringo_tune_set_cache(path: str | None) -> None:
    """Keep tuned choices in this JSON file (read now, rewritten on change)."""
    _check(load().ringo_tune_set_cache(path.encode() if path else None), "ringo_tune_set_cache")


def ringo_sort_opts_force(opts: dict | None) -> None:
    """Force radix pass options for every conversion (None: back to the
    recorded choices)."""
    if opts is None:
        _check(load().ringo_sort_opts_force(None), "ringo_sort_opts_force")
        return
    o = SortOpts(int(opts.get("rank_method", 0)), int(opts.get("prefetch_waves", 1)),
                 int(opts.get("wave_rows", 0)), int(opts.get("in_digit_bits", 8)), 0)
    _check(load().ringo_sort_opts_force(ctypes.byref(o)), "ringo_sort_opts_force")


def ringo_test_inject_alloc_failure(skip: int) -> None:
    """Test hook: the device allocation after the next `skip` ones fails
    (skip < 0 disarms)."""
    _check(load().ringo_test_inject_alloc_failure(int(skip)), "ringo_test_inject_alloc_failure")


def ringo_test_inject_lookback_timeout(spin_limit: int) -> None:
    """Test hook: the next conversion's waits are bounded by `spin_limit`
    spins and its first radix pass leaves tile 0 unclaimed."""
    _check(load().ringo_test_inject_lookback_timeout(int(spin_limit)),
           "ringo_test_inject_lookback_timeout")


def ringo_test_pool_used() -> int:
    """Test hook: bytes allocated from the library's device pool now."""
    v = ctypes.c_uint64()
    _check(load().ringo_test_pool_used(ctypes.byref(v)), "ringo_test_pool_used")
    return v.value


def ringo_version() -> str:
    return load().ringo_version().decode()


NOALLOC_MAX_ROWS = 1 << 20


def ringo_table_to_graph_noalloc(src: torch.Tensor, dst: torch.Tensor, out: dict,
                                 stream=None) -> tuple[int, int]:
    """The conversion into caller-owned device buffers, with no device
    allocation inside the library (fixed internal scratch; at most
    NOALLOC_MAX_ROWS rows; overlapping calls race).  ``out`` holds int32
    ``node_ids`` / ``out_nbr`` / ``in_nbr`` and int64 ``out_off`` / ``in_off``
    CUDA tensors.  Returns (num_nodes, num_edges)."""
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    n = src.numel()
    want = {"node_ids": torch.int32, "out_off": torch.int64, "out_nbr": torch.int32,
            "in_off": torch.int64, "in_nbr": torch.int32}
    for name, dtype in want.items():
        t = out.get(name)
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype \
                or not t.is_contiguous():
            raise ValueError(f"out[{name!r}] must be a contiguous CUDA {dtype} tensor")
    node_cap = out["node_ids"].numel()
    if min(out["out_off"].numel(), out["in_off"].numel()) < node_cap + 1:
        raise ValueError("out_off and in_off need node_ids.numel() + 1 entries")
    v = ctypes.c_int64()
    e = ctypes.c_int64()
    _check(load().ringo_table_to_graph_noalloc(
        _col_ptr(src, "src") if n else None, _col_ptr(dst, "dst") if n else None, n,
        _stream_ptr(stream), out["node_ids"].data_ptr(), out["out_off"].data_ptr(),
        out["out_nbr"].data_ptr(), out["in_off"].data_ptr(), out["in_nbr"].data_ptr(),
        node_cap, min(out["out_nbr"].numel(), out["in_nbr"].numel()),
        ctypes.byref(v), ctypes.byref(e)), "ringo_table_to_graph_noalloc")
    return v.value, e.value


# ------------------------------------------------------------ batches ------
class SelectC(ctypes.Structure):
    _fields_ = [("tags", ctypes.POINTER(ctypes.c_int32)), ("ntags", ctypes.c_int32),
                ("t0", ctypes.c_int64), ("t1", ctypes.c_int64)]


def _preds_c(preds):
    """Marshal [(tags, t0, t1), ...] into a ringo_select array (kept alive by
    the returned tuple)."""
    keep = []
    arr = (SelectC * max(1, len(preds)))()
    for i, (tags, t0, t1) in enumerate(preds):
        t = np.ascontiguousarray(np.asarray(tags, np.int32))
        keep.append(t)
        arr[i].tags = t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        arr[i].ntags = t.size
        arr[i].t0 = int(t0)
        arr[i].t1 = int(t1)
    return arr, keep


class BaseTable:
    """A resident base table (src, dst, ts, tag) clustered by (tag, ts)."""

    def __init__(self, src: torch.Tensor, dst: torch.Tensor, ts: torch.Tensor, tag: torch.Tensor,
                 stream=None):
        n = src.numel()
        if not (dst.numel() == ts.numel() == tag.numel() == n):
            raise ValueError("columns differ in length")
        if ts.dtype != torch.int64 or not ts.is_cuda:
            raise ValueError("ts must be a CUDA int64 tensor")
        h = ctypes.c_void_p()
        _check(load().ringo_base_table_load(
            _col_ptr(src, "src") if n else None, _col_ptr(dst, "dst") if n else None,
            ts.data_ptr() if n else None, _col_ptr(tag, "tag") if n else None, n,
            _stream_ptr(stream), ctypes.byref(h)), "ringo_base_table_load")
        self._h = h
        self.nrows = n

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ringo_base_table_free(self._h)
            self._h = ctypes.c_void_p(0)

    def select_count(self, preds, stream=None) -> np.ndarray:
        arr, keep = _preds_c(preds)
        out = np.zeros(max(1, len(preds)), np.int64)
        _check(load().ringo_select_count(self._h, arr, len(preds), _stream_ptr(stream),
                                         out.ctypes.data), "ringo_select_count")
        return out[:len(preds)]

    def select_gather(self, pred, cap: int, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        arr, keep = _preds_c([pred])
        src = torch.empty(max(1, cap), dtype=torch.int32, device="cuda")
        dst = torch.empty(max(1, cap), dtype=torch.int32, device="cuda")
        n = ctypes.c_int64()
        _check(load().ringo_select_gather(self._h, arr, src.data_ptr(), dst.data_ptr(), cap,
                                          ctypes.byref(n), _stream_ptr(stream)),
               "ringo_select_gather")
        return src[:n.value], dst[:n.value]

    def autotune(self, preds, stream=None) -> tuple[int, float]:
        """Times candidate wave sizes on these predicates; later convert_batch
        calls with wave_rows=0 use the fastest.  Returns (wave_rows, ms)."""
        arr, keep = _preds_c(preds)
        w = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(load().ringo_batch_autotune(self._h, arr, len(preds), _stream_ptr(stream),
                                           ctypes.byref(w), ctypes.byref(ms)),
               "ringo_batch_autotune")
        return w.value, ms.value

    def convert_batch(self, preds, wave_rows: int = 0, stream=None) -> "Batch":
        arr, keep = _preds_c(preds)
        h = ctypes.c_void_p()
        _check(load().ringo_convert_batch(self._h, arr, len(preds), int(wave_rows),
                                          _stream_ptr(stream), ctypes.byref(h)),
               "ringo_convert_batch")
        return Batch(h.value)


class Batch:
    """Owner of a ringo_batch*: one graph per predicate."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ringo_batch_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __len__(self) -> int:
        n = ctypes.c_int32()
        _check(load().ringo_batch_num_graphs(self._h, ctypes.byref(n)), "ringo_batch_num_graphs")
        return n.value

    def info(self, i: int) -> dict:
        gi = GraphInfo()
        _check(load().ringo_batch_graph_info(self._h, i, ctypes.byref(gi)),
               "ringo_batch_graph_info")
        return {f: getattr(gi, f) for f, _ in GraphInfo._fields_}

    def copy_to_host(self, i: int) -> dict:
        inf = self.info(i)
        V, E = inf["num_nodes"], inf["num_edges"]
        out = {"node_ids": np.empty(V, np.int32), "out_off": np.empty(V + 1, np.int64),
               "out_nbr": np.empty(E, np.int32), "in_off": np.empty(V + 1, np.int64),
               "in_nbr": np.empty(E, np.int32)}
        _check(load().ringo_batch_copy_graph_to_host(
            self._h, i, out["node_ids"].ctypes.data, out["out_off"].ctypes.data,
            out["out_nbr"].ctypes.data, out["in_off"].ctypes.data, out["in_nbr"].ctypes.data),
            "ringo_batch_copy_graph_to_host")
        out["num_nodes"], out["num_edges"] = V, E
        return out

    def to_edge_table(self, i: int, direction: int = RINGO_OUT,
                      stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """Edge table of graph i (as Graph.to_edge_table)."""
        E = self.info(i)["num_edges"]
        src = torch.empty(max(E, 1), dtype=torch.int32, device="cuda")
        dst = torch.empty(max(E, 1), dtype=torch.int32, device="cuda")
        n = ctypes.c_int64()
        _check(load().ringo_batch_graph_to_edge_table(self._h, i, direction, src.data_ptr(),
                                                      dst.data_ptr(), E, ctypes.byref(n),
                                                      _stream_ptr(stream)),
               "ringo_batch_graph_to_edge_table")
        return src[:n.value], dst[:n.value]

    def degree_topk(self, i: int, direction: int, k: int) -> tuple[np.ndarray, np.ndarray]:
        ids = np.zeros(max(k, 1), np.int32)
        degs = np.zeros(max(k, 1), np.int64)
        n = ctypes.c_int32()
        _check(load().ringo_batch_degree_topk(self._h, i, direction, int(k), ids.ctypes.data,
                                              degs.ctypes.data, ctypes.byref(n)),
               "ringo_batch_degree_topk")
        return ids[:n.value].copy(), degs[:n.value].copy()


# ------------------------------------------------------------- serving -----
RINGO_SERVE_KEEP_GRAPH = 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_batch_rows", ctypes.c_int64), ("small_rows", ctypes.c_int64)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_requests", ctypes.c_int32),
                ("batch_rows", ctypes.c_int64), ("nrows", ctypes.c_int64),
                ("num_nodes", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("k_out", ctypes.c_int32), ("k_in", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "failed", "batches", "rows", "max_concurrent_batches",
        "inflight_bytes", "max_inflight_bytes", "pending")]


def clock_ns() -> int:
    """The monotonic clock of the server's timestamps."""
    return int(load().ringo_clock_ns())


class Server:
    """Request server over a resident BaseTable (select + convert + top-k)."""

    def __init__(self, base: BaseTable, budget_bytes: int, workers: int = 0, max_batch: int = 0,
                 max_batch_rows: int = 0, small_rows: int = 0):
        cfg = ServerConfig(workers, max_batch, max_batch_rows, small_rows)
        h = ctypes.c_void_p()
        _check(load().ringo_server_create(base._h, int(budget_bytes), ctypes.byref(cfg),
                                          ctypes.byref(h)), "ringo_server_create")
        self._h = h
        self._base = base  # the base table must outlive the server
        self._kept = set()

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ringo_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def submit(self, pred, topk: int = 100, keep_graph: bool = False) -> int:
        arr, keep = _preds_c([pred])
        t = ctypes.c_uint64()
        _check(load().ringo_server_submit(self._h, arr, int(topk),
                                          RINGO_SERVE_KEEP_GRAPH if keep_graph else 0,
                                          ctypes.byref(t)), "ringo_server_submit")
        if keep_graph:
            self._kept.add(t.value)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        """The result of a ticket as a dict (info fields, top-k lists and, for
        keep_graph requests, the graph's host arrays)."""
        lib = load()
        r = ctypes.c_void_p()
        _check(lib.ringo_server_wait(self._h, ticket, int(timeout_us), ctypes.byref(r)),
               "ringo_server_wait")
        try:
            inf = ResultInfo()
            _check(lib.ringo_result_get_info(r, ctypes.byref(inf)), "ringo_result_get_info")
            out = {f: getattr(inf, f) for f, _ in ResultInfo._fields_}
            for d, name in ((RINGO_OUT, "topk_out"), (RINGO_IN, "topk_in")):
                k = out["k_out"] if d == RINGO_OUT else out["k_in"]
                ids = np.zeros(max(k, 1), np.int32)
                degs = np.zeros(max(k, 1), np.int64)
                n = ctypes.c_int32()
                _check(lib.ringo_result_topk(r, d, ids.ctypes.data, degs.ctypes.data, k,
                                             ctypes.byref(n)), "ringo_result_topk")
                out[name] = (ids[:n.value].copy(), degs[:n.value].copy())
            out["graph"] = None
            kept = ticket in self._kept
            self._kept.discard(ticket)
            if kept and out["status"] == RINGO_OK:
                V, E = out["num_nodes"], out["num_edges"]
                g = {"node_ids": np.empty(V, np.int32), "out_off": np.empty(V + 1, np.int64),
                     "out_nbr": np.empty(E, np.int32), "in_off": np.empty(V + 1, np.int64),
                     "in_nbr": np.empty(E, np.int32)}
                rc = lib.ringo_result_copy_graph_to_host(
                    r, g["node_ids"].ctypes.data, g["out_off"].ctypes.data,
                    g["out_nbr"].ctypes.data, g["in_off"].ctypes.data, g["in_nbr"].ctypes.data)
                if rc == RINGO_OK:
                    g["num_nodes"], g["num_edges"] = V, E
                    out["graph"] = g
            return out
        finally:
            lib.ringo_result_free(r)

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().ringo_server_get_stats(self._h, ctypes.byref(st)), "ringo_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}


# ---------------------------------------------------------- select / join --
RINGO_CMP_LT, RINGO_CMP_LE, RINGO_CMP_EQ, RINGO_CMP_NE, RINGO_CMP_GE, RINGO_CMP_GT = range(6)
_CMP = {"<": RINGO_CMP_LT, "<=": RINGO_CMP_LE, "==": RINGO_CMP_EQ, "!=": RINGO_CMP_NE,
        ">=": RINGO_CMP_GE, ">": RINGO_CMP_GT}


def ringo_table_select(src: torch.Tensor, dst: torch.Tensor, col: int, op: str, value: int,
                       stream=None) -> int:
    """Select in place on device columns; returns the number of rows kept
    (the first n rows of src and dst)."""
    n = ctypes.c_int64()
    _check(load().ringo_table_select(_col_ptr(src, "src") if src.numel() else None,
                                     _col_ptr(dst, "dst") if dst.numel() else None, src.numel(),
                                     int(col), _CMP[op], int(value), ctypes.byref(n),
                                     _stream_ptr(stream)), "ringo_table_select")
    return n.value


def ringo_table_join(src: torch.Tensor, dst: torch.Tensor, col: int, keys: torch.Tensor,
                     cap: int | None = None, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Join on column col with a single-column table of keys (device int32);
    returns the output columns."""
    if cap is None:
        cap = src.numel() * max(1, keys.numel())
        cap = min(cap, 2**31 - 1)
    # size first with a zero-capacity call, then write
    n = ctypes.c_int64()
    lib = load()
    sp = _stream_ptr(stream)
    args = (_col_ptr(src, "src") if src.numel() else None, _col_ptr(dst, "dst") if dst.numel() else None,
            src.numel(), int(col), _col_ptr(keys, "keys") if keys.numel() else None, keys.numel())
    rc = lib.ringo_table_join(*args, None, None, 0, ctypes.byref(n), sp)
    if rc not in (RINGO_OK, RINGO_ERANGE):
        _check(rc, "ringo_table_join")
    rows = n.value
    out_s = torch.empty(max(rows, 1), dtype=torch.int32, device="cuda")
    out_d = torch.empty(max(rows, 1), dtype=torch.int32, device="cuda")
    if rows:
        _check(lib.ringo_table_join(*args, out_s.data_ptr(), out_d.data_ptr(), rows,
                                    ctypes.byref(n), sp), "ringo_table_join")
    return out_s[:rows], out_d[:rows]
