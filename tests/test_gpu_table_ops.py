"""Select (in place) and join through the C ABI, against the oracle row by
row (the relational operations before conversion; Section 3.3 and Section
4's select/join benchmark)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def gpu_select(s, d, col, op, value):
    ts = torch.as_tensor(np.ascontiguousarray(s, np.int32)).cuda()
    td = torch.as_tensor(np.ascontiguousarray(d, np.int32)).cuda()
    n = ringo.ringo_table_select(ts, td, col, op, value)
    return ts[:n].cpu().numpy(), td[:n].cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 100_003, 1_000_001])
def test_select_sizes(n):
    s, d = tg.signed_table(n, max(2, n // 3), seed=n)
    s, d = s.numpy(), d.numpy()
    for col in (0, 1):
        v = int(np.median(d if col else s))
        for op in ("<", "<=", "==", "!=", ">=", ">"):
            got = gpu_select(s, d, col, op, v)
            want = oracle.table_select(s, d, col, op, v)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (col, op)


def test_select_extremes():
    s, d = tg.signed_table(50_000, 9_000, seed=3)
    s, d = s.numpy(), d.numpy()
    for v, op in ((-2**31, "<"), (2**31 - 1, "<="), (-2**31, ">="), (2**31 - 1, ">")):
        got = gpu_select(s, d, 0, op, v)
        want = oracle.table_select(s, d, 0, op, v)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("n,nk", [(1, 1), (4097, 10), (200_003, 1_000), (1_000_001, 50_000)])
def test_join_sizes(n, nk):
    sp = tg.SPECS["lj"].scaled(n)
    s, d = tg.make_table(sp, seed=n + 1)
    s, d = s.numpy(), d.numpy()
    rng = np.random.default_rng(nk)
    for col in (0, 1):
        pool = d if col else s
        keys = np.concatenate([rng.choice(pool, nk), rng.integers(-2**31, 2**31 - 1, 5)]).astype(np.int32)
        ts, td = torch.as_tensor(s).cuda(), torch.as_tensor(d).cuda()
        gs, gd = ringo.ringo_table_join(ts, td, col, torch.as_tensor(keys).cuda())
        ws, wd = oracle.table_join(s, d, col, keys)
        assert np.array_equal(gs.cpu().numpy(), ws) and np.array_equal(gd.cpu().numpy(), wd)


def test_join_cap_too_small_writes_nothing():
    import ctypes
    s = torch.arange(100, dtype=torch.int32, device="cuda")
    keys = torch.tensor([5, 5, 7], dtype=torch.int32, device="cuda")
    out = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64()
    rc = ringo.load().ringo_table_join(s.data_ptr(), s.data_ptr(), 100, 0, keys.data_ptr(), 3,
                                       out.data_ptr(), out.data_ptr(), 2, ctypes.byref(n), None)
    assert rc == ringo.RINGO_ERANGE and n.value == 3
    assert out.tolist() == [-1, -1]


def test_select_then_convert_matches_oracle():
    # the relational step feeding the conversion
    s, d = tg.make_table(tg.SPECS["twitter"].scaled(600_000), seed=9)
    s, d = s.numpy(), d.numpy()
    v = int(np.percentile(s, 30))
    ts, td = torch.as_tensor(s).cuda(), torch.as_tensor(d).cuda()
    n = ringo.ringo_table_select(ts, td, 0, "<", v)
    g = ringo.ringo_table_to_graph(ts[:n].contiguous(), td[:n].contiguous())
    got = g.copy_to_host()
    g.free()
    want = oracle.table_to_graph(*oracle.table_select(s, d, 0, "<", v))
    for k in ("node_ids", "out_off", "out_nbr", "in_off", "in_nbr"):
        assert np.array_equal(got[k], want[k])
