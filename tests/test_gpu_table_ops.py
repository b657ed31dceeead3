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


def gpu_join(s, d, col, keys):
    ts, td = torch.as_tensor(np.ascontiguousarray(s, np.int32)).cuda(), \
        torch.as_tensor(np.ascontiguousarray(d, np.int32)).cuda()
    gs, gd = ringo.ringo_table_join(ts, td, col, torch.as_tensor(np.ascontiguousarray(keys, np.int32)).cuda())
    return gs.cpu().numpy(), gd.cpu().numpy()


@pytest.mark.parametrize("dups", [False, True])
def test_join_bitmap_key_set(dups):
    # 700K keys in a 10M-wide range: the bitmap is smaller than the hash table,
    # so the key set is a bitmap (plus a hash table of repeated keys' counts);
    # rows just outside the range and at both ends of it
    rng = np.random.default_rng(11 + dups)
    keys = rng.choice(np.arange(-5_000_000, 5_000_001, dtype=np.int32), 700_000, replace=False)
    keys[:2] = (-5_000_000, 5_000_000)
    if dups:
        keys = np.concatenate([keys, keys[1000:1500], keys[1000:1100], keys[:1]])
    n = 1_000_003
    s = rng.integers(-6_000_000, 6_000_000, n).astype(np.int32)
    d = rng.integers(-6_000_000, 6_000_000, n).astype(np.int32)
    s[:4] = (-5_000_001, -5_000_000, 5_000_000, 5_000_001)
    d[-4:] = (-5_000_001, -5_000_000, 5_000_000, 5_000_001)
    s[100:200] = keys[1000:1100]  # keys met up to three times
    for col in (0, 1):
        gs, gd = gpu_join(s, d, col, keys)
        ws, wd = oracle.table_join(s, d, col, keys)
        assert np.array_equal(gs, ws) and np.array_equal(gd, wd), col


def test_join_large_hash_key_set_full_range():
    # 1.2M keys over the whole int32 range (a bitmap would be larger than the
    # hash table), both extremes among the keys and the rows
    rng = np.random.default_rng(12)
    keys = rng.integers(-2**31, 2**31 - 1, 1_200_000, dtype=np.int64).astype(np.int32)
    keys[:2] = (-2**31, 2**31 - 1)
    n = 600_001
    s = np.concatenate([rng.choice(keys, n // 2), rng.integers(-2**31, 2**31 - 1, n - n // 2)]).astype(np.int32)
    rng.shuffle(s)
    s[:2] = (-2**31, 2**31 - 1)
    d = rng.integers(-2**31, 2**31 - 1, n).astype(np.int32)
    gs, gd = gpu_join(s, d, 0, keys)
    ws, wd = oracle.table_join(s, d, 0, keys)
    assert np.array_equal(gs, ws) and np.array_equal(gd, wd)


@pytest.mark.parametrize("nk,spread", [(300, 1 << 22), (1_000_000, 1 << 22), (1_000_000, 1 << 31)])
def test_join_many_tiles(nk, spread):
    # 20M rows = 4883 tiles, so the scan of tile counts spans two blocks; the
    # three key-set forms: 300 keys (shared-memory table), 1M keys within a
    # 4M-wide range (bitmap), 1M keys over the whole range (hash table)
    rng = np.random.default_rng(nk + spread)
    ids = rng.choice(spread, 2_000_000, replace=False).astype(np.int64) - spread // 2
    s = rng.choice(ids, 20_000_000).astype(np.int32)
    d = rng.choice(ids, 20_000_000).astype(np.int32)
    keys = np.concatenate([rng.choice(ids, nk, replace=False), rng.choice(ids, nk // 100)]).astype(np.int32)
    gs, gd = gpu_join(s, d, 0, keys)
    ws, wd = oracle.table_join(s, d, 0, keys)
    assert np.array_equal(gs, ws) and np.array_equal(gd, wd)


def test_join_cap_too_small_writes_nothing_bitmap():
    import ctypes
    keys = torch.arange(0, 1_400_000, 2, dtype=torch.int32, device="cuda")  # bitmap key set
    s = torch.arange(2_000_000, dtype=torch.int32, device="cuda")
    out = torch.full((10,), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64()
    rc = ringo.load().ringo_table_join(s.data_ptr(), s.data_ptr(), s.numel(), 0, keys.data_ptr(),
                                       keys.numel(), out.data_ptr(), out.data_ptr(), 10,
                                       ctypes.byref(n), None)
    assert rc == ringo.RINGO_ERANGE and n.value == 700_000
    assert out.tolist() == [-1] * 10


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


def test_empty_inputs():
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    s = torch.arange(10, dtype=torch.int32, device="cuda")
    assert ringo.ringo_table_select(e, e.clone(), 0, "<", 5) == 0
    gs, gd = ringo.ringo_table_join(e, e.clone(), 0, torch.tensor([1, 2], dtype=torch.int32, device="cuda"))
    assert gs.numel() == 0 and gd.numel() == 0
    gs, gd = ringo.ringo_table_join(s, s.clone(), 1, e)  # no keys: nothing matches
    assert gs.numel() == 0 and gd.numel() == 0
    # nothing kept / everything kept
    t = s.clone()
    assert ringo.ringo_table_select(t, s.clone(), 0, ">", 100) == 0
    t, u = s.clone(), s.clone() * 2
    assert ringo.ringo_table_select(t, u, 1, ">=", 0) == 10
    assert torch.equal(t, s) and torch.equal(u, s * 2)
