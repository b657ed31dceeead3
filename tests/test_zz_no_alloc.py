"""The allocation-free entry point, for callers that cannot allocate device
memory when they convert a table (a budget reserved up front, a serving loop
that must not enter the allocator).  Its output must equal that of the
regular entry point, exactly (integer results), on consecutive calls that
share the library's fixed scratch array.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def _noalloc_call(src, dst):
    """Call the C ABI directly with caller-owned output buffers."""
    lib = ringo.load()
    n = src.numel()
    cap_v = max(1, 2 * n)
    bufs = {"node_ids": torch.full((cap_v,), -7, dtype=torch.int32, device="cuda"),
            "out_off": torch.full((cap_v + 1,), -7, dtype=torch.int64, device="cuda"),
            "out_nbr": torch.full((max(1, n),), -7, dtype=torch.int32, device="cuda"),
            "in_off": torch.full((cap_v + 1,), -7, dtype=torch.int64, device="cuda"),
            "in_nbr": torch.full((max(1, n),), -7, dtype=torch.int32, device="cuda")}
    v, e = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.ringo_table_to_graph_noalloc(
        src.data_ptr() if n else None, dst.data_ptr() if n else None, n,
        torch.cuda.current_stream().cuda_stream, bufs["node_ids"].data_ptr(),
        bufs["out_off"].data_ptr(), bufs["out_nbr"].data_ptr(), bufs["in_off"].data_ptr(),
        bufs["in_nbr"].data_ptr(), cap_v, max(1, n), ctypes.byref(v), ctypes.byref(e))
    assert rc == ringo.RINGO_OK, lib.ringo_last_error()
    V, E = v.value, e.value
    return {"num_nodes": V, "num_edges": E,
            "node_ids": bufs["node_ids"][:V].cpu().numpy(),
            "out_off": bufs["out_off"][:V + 1].cpu().numpy(),
            "out_nbr": bufs["out_nbr"][:E].cpu().numpy(),
            "in_off": bufs["in_off"][:V + 1].cpu().numpy(),
            "in_nbr": bufs["in_nbr"][:E].cpu().numpy()}


def _regular(src, dst):
    g = ringo.ringo_table_to_graph(src, dst)
    a = g.copy_to_host()
    g.free()
    return a


def _same(a, b):
    assert a["num_nodes"] == b["num_nodes"] and a["num_edges"] == b["num_edges"]
    for k in ("node_ids", "out_off", "out_nbr", "in_off", "in_nbr"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_noalloc_matches_regular_entry_twice_in_a_row():
    t1 = tg.make_table(tg.SPECS["twitter"].scaled(700_000), seed=21, device="cuda")
    t2 = tg.signed_table(ringo.NOALLOC_MAX_ROWS, 150_000, seed=22, device="cuda")
    for src, dst in (t1, t2, t1):
        _same(_noalloc_call(src, dst), _regular(src, dst))


def test_noalloc_limits_and_empty():
    lib = ringo.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    v, e = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.ringo_table_to_graph_noalloc(fake, fake, ringo.NOALLOC_MAX_ROWS + 1, None, fake,
                                          fake, fake, fake, fake, 1 << 30, 1 << 30,
                                          ctypes.byref(v), ctypes.byref(e))
    assert rc == ringo.RINGO_ERANGE
    assert b"RINGO_NOALLOC_MAX_ROWS" in lib.ringo_last_error()
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    a = _noalloc_call(empty, empty)
    assert a["num_nodes"] == 0 and a["num_edges"] == 0
    assert a["out_off"].tolist() == [0] and a["in_off"].tolist() == [0]


def test_noalloc_node_capacity_error_then_next_call_unaffected():
    """node_capacity is checked after the sort, once the distinct source and
    destination counts are known; the call has written scratch and the
    neighbour buffers by then, and the next call must not notice."""
    lib = ringo.load()
    src, dst = tg.make_table(tg.SPECS["tiny"].scaled(20_000), seed=31, device="cuda")
    n = src.numel()
    bufs = [torch.empty(k, dtype=t, device="cuda") for k, t in
            ((1, torch.int32), (2, torch.int64), (n, torch.int32), (2, torch.int64),
             (n, torch.int32))]
    v, e = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.ringo_table_to_graph_noalloc(
        src.data_ptr(), dst.data_ptr(), n, torch.cuda.current_stream().cuda_stream,
        *[b.data_ptr() for b in bufs], 1, n, ctypes.byref(v), ctypes.byref(e))
    assert rc == ringo.RINGO_ERANGE
    assert b"node_capacity" in lib.ringo_last_error()
    s2, d2 = tg.signed_table(300_000, 40_000, seed=32, device="cuda")
    _same(_noalloc_call(s2, d2), _regular(s2, d2))


def test_noalloc_python_wrapper():
    """The same entry point through the binding, with its argument checks."""
    src, dst = tg.make_table(tg.SPECS["lj"].scaled(250_000), seed=33, device="cuda")
    n = src.numel()
    out = {"node_ids": torch.empty(2 * n, dtype=torch.int32, device="cuda"),
           "out_off": torch.empty(2 * n + 1, dtype=torch.int64, device="cuda"),
           "out_nbr": torch.empty(n, dtype=torch.int32, device="cuda"),
           "in_off": torch.empty(2 * n + 1, dtype=torch.int64, device="cuda"),
           "in_nbr": torch.empty(n, dtype=torch.int32, device="cuda")}
    V, E = ringo.ringo_table_to_graph_noalloc(src, dst, out)
    got = {"num_nodes": V, "num_edges": E,
           "node_ids": out["node_ids"][:V].cpu().numpy(),
           "out_off": out["out_off"][:V + 1].cpu().numpy(),
           "out_nbr": out["out_nbr"][:E].cpu().numpy(),
           "in_off": out["in_off"][:V + 1].cpu().numpy(),
           "in_nbr": out["in_nbr"][:E].cpu().numpy()}
    _same(got, _regular(src, dst))
    short = dict(out, out_off=out["out_off"][:2 * n])  # one entry short
    with pytest.raises(ValueError):
        ringo.ringo_table_to_graph_noalloc(src, dst, short)
    wrong = dict(out, in_nbr=out["in_nbr"].to(torch.int64))
    with pytest.raises(ValueError):
        ringo.ringo_table_to_graph_noalloc(src, dst, wrong)
