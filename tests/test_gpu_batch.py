"""Base tables, selection and batched conversion through the C ABI.

Every graph of a batch is compared element by element with the oracle run on
the same rows, selected on the host with numpy from the original (unclustered)
columns: the batch must equal the conversion of each selection alone
(Section 3.4 applied to the sub-table a Section 3.3 select produces).
"""
import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def host_select(cols, pred):
    src, dst, ts, tag = cols
    tags, t0, t1 = pred
    m = np.isin(tag, np.asarray(tags, np.int32)) & (ts >= t0) & (ts < t1)
    return src[m], dst[m]


def load(cols):
    src, dst, ts, tag = (torch.as_tensor(np.ascontiguousarray(c)).cuda() for c in cols)
    return ringo.BaseTable(src, dst, ts, tag)


def check_batch(base, cols, preds, wave_rows=0):
    bt = base.convert_batch(preds, wave_rows=wave_rows)
    try:
        assert len(bt) == len(preds)
        counts = base.select_count(preds)
        for i, p in enumerate(preds):
            s, d = host_select(cols, p)
            assert counts[i] == s.size, f"pred {i}: count"
            inf = bt.info(i)
            assert inf["nrows"] == s.size
            want = oracle.table_to_graph(s, d)
            got = bt.copy_to_host(i)
            pins.assert_same_graph(got, want, f"pred {i} ({s.size} rows)")
            assert inf["num_src_nodes"] == np.unique(s).size
            assert inf["num_dst_nodes"] == np.unique(d).size
    finally:
        bt.free()


def ragged_base(seed=11):
    """Tag k holds a signed-ID table of sizes[k] rows; ts uniform in [0, 1000)."""
    sizes = [1, 2, 31, 4095, 4096, 4097, 12289, 65537, 3, 200_003]
    parts = []
    for k, n in enumerate(sizes):
        s, d = tg.signed_table(n, max(2, n // 7), seed=seed + k)
        parts.append((s.numpy(), d.numpy(), np.full(n, k + 1, np.int32)))
    src = np.concatenate([p[0] for p in parts])
    dst = np.concatenate([p[1] for p in parts])
    tag = np.concatenate([p[2] for p in parts])
    rng = np.random.default_rng(seed)
    ts = rng.integers(0, 1000, src.size).astype(np.int64)
    order = rng.permutation(src.size)  # tags interleaved in the base table
    return src[order], dst[order], ts[order], tag[order], len(sizes)


def ragged_preds(ntags):
    preds = [([k], 0, 1000) for k in range(1, ntags + 1)]  # each tag alone
    preds += [
        ([], 0, 1000),                 # no tags
        ([3, 4], 500, 500),            # empty window
        ([999, -7], 0, 1000),          # tags not in the table
        ([5, 5, 5], 0, 1000),          # a repeated tag counts once
        ([2, 8, 6], 100, 900),         # several tags, part of the window
        ([8], -10**12, 10**12),        # window wider than the table
        ([8], 999, 1000),              # one time step
        (list(range(1, ntags + 1)), 250, 750),
        ([10, 7], 0, 1000),
    ]
    return preds


def test_ragged_batch_default_wave():
    src, dst, ts, tag, nt = ragged_base()
    cols = (src, dst, ts, tag)
    base = load(cols)
    try:
        check_batch(base, cols, ragged_preds(nt))
    finally:
        base.free()


def test_ragged_batch_many_waves():
    src, dst, ts, tag, nt = ragged_base(seed=21)
    cols = (src, dst, ts, tag)
    base = load(cols)
    try:
        check_batch(base, cols, ragged_preds(nt), wave_rows=5000)
    finally:
        base.free()


def test_golden_tables_in_one_batch():
    tabs = [pins.load_golden(p) for p in pins.golden_files()]
    src = np.concatenate([t["src"] for t in tabs]).astype(np.int32)
    dst = np.concatenate([t["dst"] for t in tabs]).astype(np.int32)
    tag = np.concatenate([np.full(len(t["src"]), k, np.int32) for k, t in enumerate(tabs)])
    ts = np.zeros(src.size, np.int64)
    cols = (src, dst, ts, tag)
    base = load(cols)
    try:
        bt = base.convert_batch([([k], 0, 1) for k in range(len(tabs))])
        for k, t in enumerate(tabs):
            pins.assert_same_graph(bt.copy_to_host(k), t, f"golden {k}")
        bt.free()
    finally:
        base.free()


def test_select_count_and_gather():
    sp = tg.BaseSpec(rows=1_000_003, nodes=80_000, tags=300)
    cols = tuple(c.numpy() for c in tg.make_base_table(sp, seed=5))
    base = load(cols)
    try:
        preds = tg.make_predicates(sp, 40, 100, 200_000, seed=3)
        counts = base.select_count(preds)
        for i, p in enumerate(preds):
            s, d = host_select(cols, p)
            assert counts[i] == s.size
            gs, gd = base.select_gather(p, cap=s.size)
            got = np.sort(gs.cpu().numpy().astype(np.int64) << 32
                          | (gd.cpu().numpy().astype(np.int64) & 0xFFFFFFFF))
            want = np.sort(s.astype(np.int64) << 32 | (d.astype(np.int64) & 0xFFFFFFFF))
            assert np.array_equal(got, want), f"pred {i}: gathered rows"
        if counts.max() > 0:
            with pytest.raises(ringo.RingoError) as e:
                base.select_gather(preds[int(np.argmax(counts))], cap=int(counts.max()) - 1)
            assert e.value.status == ringo.RINGO_ERANGE
    finally:
        base.free()


def test_clustered_order():
    # gather returns each tag's rows in ts order; one tag per predicate
    sp = tg.BaseSpec(rows=300_000, nodes=30_000, tags=20)
    src, dst, ts, tag = (c.numpy() for c in tg.make_base_table(sp, seed=9))
    # encode the row index in src so the gathered order can be read back
    src = np.arange(src.size, dtype=np.int32)
    cols = (src, dst, ts, tag)
    base = load(cols)
    try:
        for t in (0, 3, 19):
            gs, _ = base.select_gather(([t], tg.TS0, tg.TS0 + tg.FIVE_YEARS), cap=sp.rows)
            rows = gs.cpu().numpy()
            want = np.flatnonzero(tag == t)
            want = want[np.argsort(ts[want], kind="stable")]
            assert np.array_equal(rows, want)
    finally:
        base.free()


def test_scaled_batch_matches_oracle():
    sp = tg.BaseSpec(rows=3_000_000, nodes=240_000, tags=400)
    cols = tuple(c.numpy() for c in tg.make_base_table(sp, seed=2))
    base = load(cols)
    try:
        preds = tg.make_predicates(sp, 48, 1000, 300_000, seed=4)
        check_batch(base, cols, preds)
    finally:
        base.free()


def test_batch_degree_topk():
    sp = tg.BaseSpec(rows=500_000, nodes=40_000, tags=50)
    cols = tuple(c.numpy() for c in tg.make_base_table(sp, seed=8))
    base = load(cols)
    try:
        preds = tg.make_predicates(sp, 6, 5_000, 200_000, seed=8)
        bt = base.convert_batch(preds)
        for i, p in enumerate(preds):
            want = oracle.table_to_graph(*host_select(cols, p))
            ids = want["node_ids"]
            for di, name in ((0, "out"), (1, "in")):
                deg = np.diff(want[f"{name}_off"])
                for k in (1, 100):
                    tid, tdeg = bt.degree_topk(i, di, k)
                    order = np.lexsort((ids, -deg))[:k]
                    assert np.array_equal(tid, ids[order]) and np.array_equal(tdeg, deg[order])
        bt.free()
    finally:
        base.free()


def test_empty_base_and_empty_batch():
    e32 = np.zeros(0, np.int32)
    cols = (e32, e32, np.zeros(0, np.int64), e32)
    base = ringo.BaseTable(*(torch.as_tensor(c).cuda() for c in cols))
    try:
        bt = base.convert_batch([([1], 0, 10), ([], 0, 0)])
        for i in range(2):
            g = bt.copy_to_host(i)
            assert g["num_nodes"] == 0 and g["num_edges"] == 0
            assert g["out_off"].tolist() == [0] and g["in_off"].tolist() == [0]
        bt.free()
        bt = base.convert_batch([])
        assert len(bt) == 0
        bt.free()
    finally:
        base.free()


def test_ts_range_rejected():
    src = np.zeros(2, np.int32)
    ts = np.array([0, 1 << 32], np.int64)
    with pytest.raises(ringo.RingoError) as e:
        load((src, src, ts, src))
    assert e.value.status == ringo.RINGO_ERANGE


def test_autotune_then_batch():
    sp = tg.BaseSpec(rows=1_500_000, nodes=120_000, tags=200)
    cols = tuple(c.numpy() for c in tg.make_base_table(sp, seed=6))
    base = load(cols)
    try:
        preds = tg.make_predicates(sp, 24, 1_000, 200_000, seed=6)
        w, ms = base.autotune(preds)
        assert w >= 1 and ms > 0
        check_batch(base, cols, preds)  # wave_rows=0 takes the tuned size
    finally:
        base.free()
