"""Graph -> table (Section 3.4, "Conversion of graphs to tables") through the
C ABI: edge tables in both CSR orders and the node table, against the closed
form (the table's distinct rows), against the oracle element by element, and
by round trip at full size."""
import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def gpu_tables(src, dst) -> dict:
    s = torch.as_tensor(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.as_tensor(np.ascontiguousarray(dst, np.int32)).cuda()
    g = ringo.ringo_table_to_graph(s, d)
    try:
        os_, od = g.to_edge_table(ringo.RINGO_OUT)
        is_, id_ = g.to_edge_table(ringo.RINGO_IN)
        ids, outdeg, indeg = g.to_node_table()
        torch.cuda.synchronize()
        return {"out_src": os_.cpu().numpy(), "out_dst": od.cpu().numpy(),
                "in_src": is_.cpu().numpy(), "in_dst": id_.cpu().numpy(),
                "ids": ids.cpu().numpy(), "outdeg": outdeg.cpu().numpy(),
                "indeg": indeg.cpu().numpy()}
    finally:
        g.free()


def oracle_tables(src, dst) -> dict:
    g = oracle.table_to_graph(src, dst)
    os_, od = oracle.graph_to_edge_table(g, "out")
    is_, id_ = oracle.graph_to_edge_table(g, "in")
    ids, outdeg, indeg = oracle.graph_to_node_table(g)
    return {"out_src": os_, "out_dst": od, "in_src": is_, "in_dst": id_, "ids": ids,
            "outdeg": outdeg, "indeg": indeg}


def test_pins_on_gpu():
    pins.check_graph_to_table(gpu_tables, max_rows=2, trials=60)


@pytest.mark.parametrize("n", [1, 31, 2049, 4097, 100_003])
def test_ragged_sizes(n):
    s, d = tg.signed_table(n, max(2, n // 5), seed=n + 3)
    s, d = s.numpy(), d.numpy()
    pins.assert_same_tables(gpu_tables(s, d), oracle_tables(s, d), f"n={n}")


@pytest.mark.parametrize("spec", ["tiny", "lj", "twitter"])
def test_shapes_scaled(spec):
    sp = tg.SPECS[spec].scaled(1_200_007)
    s, d = tg.make_table(sp, seed=5)
    s, d = s.numpy(), d.numpy()
    pins.assert_same_tables(gpu_tables(s, d), oracle_tables(s, d), sp.name)


def test_many_zero_degree_nodes():
    # one source with edges to 50K destinations: 50K nodes of out-degree 0
    # after it, so edge tiles of the in-direction span wide node ranges
    d = np.arange(50_000, dtype=np.int32) * 3 + 7
    s = np.full(d.size, -5, np.int32)
    s = np.concatenate([s, d[:10]])
    d = np.concatenate([d, np.full(10, -5, np.int32)])
    pins.assert_same_tables(gpu_tables(s, d), oracle_tables(s, d), "star")


def test_lj_full_size_round_trip():
    src, dst = tg.make_table("lj", seed=1, device="cuda")
    g = ringo.ringo_table_to_graph(src, dst)
    del src, dst
    V, E = g.num_nodes, g.num_edges
    for direction in (ringo.RINGO_OUT, ringo.RINGO_IN):
        es, ed = g.to_edge_table(direction)
        assert es.numel() == E
        # rows strictly increasing in the direction's (row node, neighbour) order
        a, b = (es, ed) if direction == ringo.RINGO_OUT else (ed, es)
        # signed (a, b) order as signed 64-bit order: a in the high half, b
        # biased into an unsigned low half
        k = (a.long() << 32) | ((b.long() & 0xFFFFFFFF) ^ 0x80000000)
        assert bool((k[1:] > k[:-1]).all())
        g2 = ringo.ringo_table_to_graph(es, ed)
        assert g2.num_nodes == V and g2.num_edges == E
        assert torch.equal(g2.node_ids(), g.node_ids())
        for dd in (ringo.RINGO_OUT, ringo.RINGO_IN):
            o1, n1 = g.csr(dd)
            o2, n2 = g2.csr(dd)
            assert torch.equal(o1, o2) and torch.equal(n1, n2)
        g2.free()
        del es, ed, k
    ids, outdeg, indeg = g.to_node_table()
    assert int(outdeg.sum()) == E and int(indeg.sum()) == E
    assert bool(((outdeg + indeg) >= 1).all())
    g.free()


def test_batch_graph_edge_tables():
    sp = tg.BaseSpec(rows=400_000, nodes=30_000, tags=40)
    cols = tuple(c.numpy() for c in tg.make_base_table(sp, seed=3))
    base = ringo.BaseTable(*(torch.as_tensor(c).cuda() for c in cols))
    try:
        preds = tg.make_predicates(sp, 6, 1_000, 100_000, seed=3) + [([], 0, 1)]
        bt = base.convert_batch(preds)
        for i, (tags, t0, t1) in enumerate(preds):
            src, dst, ts, tag = cols
            m = np.isin(tag, np.asarray(tags, np.int32)) & (ts >= t0) & (ts < t1)
            want = oracle_tables(src[m], dst[m])
            for direction, name in ((ringo.RINGO_OUT, "out"), (ringo.RINGO_IN, "in")):
                es, ed = bt.to_edge_table(i, direction)
                torch.cuda.synchronize()
                assert np.array_equal(es.cpu().numpy(), want[f"{name}_src"])
                assert np.array_equal(ed.cpu().numpy(), want[f"{name}_dst"])
        bt.free()
    finally:
        base.free()


def test_cap_too_small_and_empty_graph():
    g = ringo.ringo_table_to_graph(torch.tensor([1, 2], dtype=torch.int32, device="cuda"),
                                   torch.tensor([2, 3], dtype=torch.int32, device="cuda"))
    small = (torch.empty(1, dtype=torch.int32, device="cuda"),
             torch.empty(1, dtype=torch.int32, device="cuda"))
    with pytest.raises(ringo.RingoError) as e:
        g.to_edge_table(ringo.RINGO_OUT, out=small)
    assert e.value.status == ringo.RINGO_ERANGE
    g.free()
    e32 = torch.empty(0, dtype=torch.int32, device="cuda")
    g = ringo.ringo_table_to_graph(e32, e32)
    es, ed = g.to_edge_table()
    ids, od, idg = g.to_node_table()
    assert es.numel() == 0 and ids.numel() == 0
    g.free()
