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
