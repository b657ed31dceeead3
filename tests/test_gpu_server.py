"""The request server through the C ABI: every result equals the oracle on
the same selection and equals the same request served alone; admission keeps
the bytes in flight within the budget."""
import threading

import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu

SPEC = tg.BaseSpec(rows=2_000_003, nodes=160_000, tags=300)


@pytest.fixture(scope="module")
def base_cols():
    cols = tuple(c.numpy() for c in tg.make_base_table(SPEC, seed=7))
    t = [torch.as_tensor(c).cuda() for c in cols]
    base = ringo.BaseTable(*t)
    del t
    yield base, cols
    base.free()


def host_select(cols, pred):
    src, dst, ts, tag = cols
    tags, t0, t1 = pred
    m = np.isin(tag, np.asarray(tags, np.int32)) & (ts >= t0) & (ts < t1)
    return src[m], dst[m]


def expected_topk(g, k):
    ids = g["node_ids"]
    out = {}
    for name in ("out", "in"):
        deg = np.diff(g[f"{name}_off"])
        order = np.lexsort((ids, -deg))[:k]
        out[name] = (ids[order], deg[order])
    return out


def check_result(res, cols, pred, k):
    s, d = host_select(cols, pred)
    want = oracle.table_to_graph(s, d)
    assert res["status"] == ringo.RINGO_OK
    assert res["nrows"] == s.size
    assert res["num_nodes"] == want["num_nodes"] and res["num_edges"] == want["num_edges"]
    if res["graph"] is not None:
        pins.assert_same_graph(res["graph"], want, f"served {s.size} rows")
    exp = expected_topk(want, k)
    for name in ("out", "in"):
        ids, degs = res[f"topk_{name}"]
        assert np.array_equal(ids, exp[name][0]) and np.array_equal(degs, exp[name][1])


def strip(res):
    return {k: v for k, v in res.items()
            if k not in ("t_submit_ns", "t_admit_ns", "t_done_ns", "batch_requests", "batch_rows")}


def same_result(a, b):
    a, b = strip(a), strip(b)
    assert a.keys() == b.keys()
    for k in a:
        if k == "graph":
            if a[k] is None or b[k] is None:
                assert a[k] is None and b[k] is None
            else:
                pins.assert_same_graph(a[k], b[k], "mix vs alone")
        elif k.startswith("topk"):
            assert all(np.array_equal(x, y) for x, y in zip(a[k], b[k]))
        else:
            assert a[k] == b[k], k


def test_mix_equals_alone_and_oracle(base_cols):
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 40, 1_000, 300_000, seed=12)
    preds += [([], 0, 10), ([5], tg.TS0 + 10, tg.TS0 + 10), ([10**6], 0, 1 << 40)]
    srv = ringo.Server(base, 40 << 30, workers=2)
    try:
        tickets = [srv.submit(p, topk=100, keep_graph=True) for p in preds]
        mixed = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(preds) and st["failed"] == 0
    assert st["batches"] < len(preds), "arrivals were batched"
    alone_srv = ringo.Server(base, 40 << 30, workers=1)
    try:
        for p, m in zip(preds, mixed):
            check_result(m, cols, p, 100)
            a = alone_srv.wait(alone_srv.submit(p, topk=100, keep_graph=True))
            assert a["batch_requests"] == 1
            same_result(m, a)
    finally:
        alone_srv.close()


def test_topk_only_results_match_batch(base_cols):
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 12, 5_000, 400_000, seed=13)
    srv = ringo.Server(base, 40 << 30)
    try:
        res = [srv.wait(srv.submit(p, topk=k)) for p, k in zip(preds, [1, 7, 100, 4096] * 3)]
    finally:
        srv.close()
    bt = base.convert_batch(preds)
    try:
        for i, (r, k) in enumerate(zip(res, [1, 7, 100, 4096] * 3)):
            assert r["graph"] is None
            for d, name in ((0, "out"), (1, "in")):
                ids, degs = bt.degree_topk(i, d, k)
                assert np.array_equal(r[f"topk_{name}"][0], ids)
                assert np.array_equal(r[f"topk_{name}"][1], degs)
    finally:
        bt.free()


def test_budget_admission(base_cols):
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 16, 50_000, 150_000, seed=14)
    counts = base.select_count(preds)
    # room for about two requests at a time
    budget = int(2.5 * 120 * int(counts.max())) + (8 << 20)
    srv = ringo.Server(base, budget, workers=3)
    try:
        tickets = [srv.submit(p, topk=10) for p in preds]
        big = srv.submit(([int(t) for t in range(SPEC.tags)], 0, 1 << 40), topk=10)
        res = [srv.wait(t) for t in tickets]
        rb = srv.wait(big)
        st = srv.stats()
    finally:
        srv.close()
    for p, r in zip(preds, res):
        check_result(r, cols, p, 10)
    assert rb["status"] == ringo.RINGO_ENOMEM
    assert st["max_inflight_bytes"] <= budget
    assert st["inflight_bytes"] == 0
    assert st["failed"] == 1 and st["completed"] == len(preds)


def test_kept_graph_charged_until_freed(base_cols):
    base, cols = base_cols
    pred = tg.make_predicates(SPEC, 1, 100_000, 100_001, seed=15)[0]
    srv = ringo.Server(base, 40 << 30)
    try:
        lib = ringo.load()
        import ctypes
        arr, keep = ringo._preds_c([pred])
        t = ctypes.c_uint64()
        assert lib.ringo_server_submit(srv._h, arr, 5, ringo.RINGO_SERVE_KEEP_GRAPH,
                                       ctypes.byref(t)) == 0
        r = ctypes.c_void_p()
        assert lib.ringo_server_wait(srv._h, t.value, -1, ctypes.byref(r)) == 0
        assert srv.stats()["inflight_bytes"] > 0
        lib.ringo_result_free(r)
        assert srv.stats()["inflight_bytes"] == 0
        with pytest.raises(ringo.RingoError) as e:
            srv.wait(t.value)
        assert e.value.status == ringo.RINGO_ENOTFOUND
    finally:
        srv.close()


def test_concurrent_submitters(base_cols):
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 24, 1_000, 100_000, seed=16)
    srv = ringo.Server(base, 40 << 30, workers=2)
    out = [None] * len(preds)

    def client(ix):
        for i in ix:
            out[i] = srv.wait(srv.submit(preds[i], topk=20))

    th = [threading.Thread(target=client, args=(range(j, len(preds), 4),)) for j in range(4)]
    try:
        for t in th:
            t.start()
        for t in th:
            t.join()
    finally:
        srv.close()
    for p, r in zip(preds, out):
        check_result(r, cols, p, 20)


def test_argument_errors(base_cols):
    base, _ = base_cols
    srv = ringo.Server(base, 1 << 30)
    try:
        with pytest.raises(ringo.RingoError) as e:
            srv.submit(([1], 0, 10), topk=4097)
        assert e.value.status == ringo.RINGO_ERANGE
        with pytest.raises(ringo.RingoError) as e:
            srv.wait(987654321)
        assert e.value.status == ringo.RINGO_ENOTFOUND
    finally:
        srv.close()
    with pytest.raises(ringo.RingoError) as e:
        ringo.Server(base, 0)
    assert e.value.status == ringo.RINGO_EINVAL


@pytest.mark.parametrize("small_rows", [-1, 20_000])
def test_small_lane_results_equal_alone(base_cols, small_rows):
    """With the small lane (requests of at most small_rows rows may also go
    to a worker on a high-priority stream) and without it, every result of a
    mix of small and large requests equals the oracle's and the same request
    served alone."""
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 30, 500, 400_000, seed=21)
    srv = ringo.Server(base, 40 << 30, workers=1, small_rows=small_rows)
    try:
        tickets = [srv.submit(p, topk=50) for p in preds]
        mixed = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(preds) and st["failed"] == 0
    alone = ringo.Server(base, 40 << 30, workers=1, small_rows=-1)
    try:
        for p, m in zip(preds, mixed):
            check_result(m, cols, p, 50)
            same_result(m, alone.wait(alone.submit(p, topk=50)))
    finally:
        alone.close()


def test_small_lane_with_a_tight_budget_and_mixed_sizes(base_cols):
    """Small requests of different sizes under a budget that holds only one
    or two of them, with a request larger than the whole budget in the
    middle: the small lane skips the ones that do not fit and admits later
    ones that do; everything finishes, the large one with ENOMEM."""
    base, cols = base_cols
    preds = tg.make_predicates(SPEC, 24, 20_000, 200_000, seed=31)
    counts = base.select_count(preds)
    budget = int(1.5 * 120 * int(counts.max())) + (8 << 20)
    huge = ([int(t) for t in range(SPEC.tags)], 0, 1 << 40)
    for rep in range(3):
        srv = ringo.Server(base, budget, workers=2)
        try:
            tickets = [srv.submit(p, topk=5) for p in preds[:12]]
            big = srv.submit(huge, topk=5)
            tickets += [srv.submit(p, topk=5) for p in preds[12:]]
            res = [srv.wait(t, timeout_us=120_000_000) for t in tickets]
            rb = srv.wait(big, timeout_us=120_000_000)
            st = srv.stats()
        finally:
            srv.close()
        for p, r in zip(preds, res):
            check_result(r, cols, p, 5)
        assert rb["status"] == ringo.RINGO_ENOMEM
        assert st["max_inflight_bytes"] <= budget and st["inflight_bytes"] == 0
