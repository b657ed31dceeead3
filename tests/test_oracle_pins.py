"""The oracle against things that do not depend on it (CPU only).

Pins: hand-worked golden tables, exhaustive brute force through an adjacency
matrix, invariants of any correct result, closed-form special cases, and
invariance under row order and duplicate rows.  A last test builds oracle
variants with one planted mistake each and checks that the pins catch every
one of them.
"""
import numpy as np
import pytest

import oracle
import pins
from paper_1503_07881_gb300 import tablegen as tg


def conv(s, d):
    return oracle.table_to_graph(s, d)


def test_golden_tables():
    pins.check_golden(conv)


def test_brute_force_exhaustive_small_alphabet():
    n = pins.check_brute_force_exhaustive(conv, alphabet=(-1, 0, 1, 2), max_rows=3)
    assert n == 1 + 16 + 256 + 4096


@pytest.mark.slow
def test_brute_force_exhaustive_four_rows():
    # every table of up to four rows over {-1, 0, 1}: 9**4 + ... tables
    pins.check_brute_force_exhaustive(conv, alphabet=(-1, 0, 1), max_rows=4)


def test_brute_force_random_extreme_ids():
    pins.check_brute_force_random(conv, trials=400)


def test_special_cases():
    pins.check_special_cases(conv)


@pytest.mark.parametrize("spec", ["tiny", "lj", "twitter"])
def test_invariants_generated(spec):
    sp = tg.SPECS[spec].scaled(60_000) if spec != "tiny" else tg.SPECS["tiny"].scaled(60_000)
    s, d = tg.make_table(sp, seed=3)
    s, d = s.numpy(), d.numpy()
    g = conv(s, d)
    pins.check_invariants(g, s, d)


def test_invariants_signed():
    s, d = tg.signed_table(20_000, 3_000, seed=5)
    s, d = s.numpy(), d.numpy()
    pins.check_invariants(conv(s, d), s, d)


def test_row_order_and_duplicates():
    s, d = tg.signed_table(5_000, 700, seed=9)
    pins.check_row_order_and_duplicates(conv, s.numpy(), d.numpy())


def test_sample_lists_agree_with_full():
    s, d = tg.make_table(tg.SPECS["tiny"].scaled(30_000), seed=2)
    s, d = s.numpy(), d.numpy()
    g = conv(s, d)
    ids = g["node_ids"]
    q = np.r_[ids[:5], ids[-5:], ids[len(ids) // 2], np.int32(-12345)]
    outs, ins, present = oracle.sample_lists(s, d, q)
    for k, x in enumerate(q):
        r = np.searchsorted(ids, x)
        if r < len(ids) and ids[r] == x:
            assert present[k]
            assert np.array_equal(outs[k], ids[g["out_nbr"][g["out_off"][r]:g["out_off"][r + 1]]])
            assert np.array_equal(ins[k], ids[g["in_nbr"][g["in_off"][r]:g["in_off"][r + 1]]])
        else:
            assert not present[k] and outs[k].size == 0 and ins[k].size == 0
    e, v = oracle.count_distinct(s, d)
    assert (e, v) == (g["num_edges"], g["num_nodes"])


MUTANTS = {
    1: "duplicates kept",
    2: "in-direction not transposed",
    3: "last offset off by one",
    4: "self-loops dropped",
    5: "unsigned ID order",
    6: "neighbour index shifted",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    """Each planted mistake (built on the CPU) must fail at least one pin."""
    def mconv(s, d):
        return oracle.table_to_graph(s, d, mutant=mutant)

    caught = []
    for name, fn in [
        ("golden", lambda: pins.check_golden(mconv)),
        ("brute", lambda: pins.check_brute_force_exhaustive(mconv, max_rows=2)),
        ("random", lambda: pins.check_brute_force_random(mconv, trials=100)),
        ("special", lambda: pins.check_special_cases(mconv)),
    ]:
        try:
            fn()
        except (AssertionError, IndexError, ValueError):
            caught.append(name)
    assert caught, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"


def oracle_tables(src, dst, mutant: int = 0) -> dict:
    g = oracle.table_to_graph(src, dst)
    os_, od = oracle.graph_to_edge_table(g, "out", mutant=mutant)
    is_, id_ = oracle.graph_to_edge_table(g, "in", mutant=mutant)
    ids, outdeg, indeg = oracle.graph_to_node_table(g)
    return {"out_src": os_, "out_dst": od, "in_src": is_, "in_dst": id_, "ids": ids,
            "outdeg": outdeg, "indeg": indeg}


def test_graph_to_table_pins():
    pins.check_graph_to_table(oracle_tables)


def test_graph_to_table_round_trip():
    # the edge table converts back to the same graph, in either row order
    rng = np.random.default_rng(4)
    for n in (0, 1, 17, 500):
        s = rng.integers(-50, 50, n).astype(np.int32)
        d = rng.integers(-50, 50, n).astype(np.int32)
        g = oracle.table_to_graph(s, d)
        for direction in ("out", "in"):
            pins.assert_same_graph(oracle.table_to_graph(*oracle.graph_to_edge_table(g, direction)),
                                   g, f"round trip {direction} n={n}")


@pytest.mark.parametrize("mutant", [7, 8])
def test_graph_to_table_pins_catch_planted_mistake(mutant):
    with pytest.raises(AssertionError):
        pins.check_graph_to_table(lambda s, d: oracle_tables(s, d, mutant=mutant))


# ------------------------------------------------------------- PageRank ---
def dense_pagerank(src, dst, damping=0.85, iterations=10):
    """Power iteration with the explicit V x V transition matrix (a route
    independent of the CSR): column-stochastic over out-edges, uniform
    columns for nodes without out-edges, then teleportation."""
    ids = sorted(set(int(x) for x in src) | set(int(x) for x in dst))
    idx = {x: i for i, x in enumerate(ids)}
    V = len(ids)
    A = np.zeros((V, V))
    for a, b in set(zip((int(x) for x in src), (int(x) for x in dst))):
        A[idx[b], idx[a]] = 1.0
    colsum = A.sum(axis=0)
    M = np.where(colsum > 0, A / np.maximum(colsum, 1), 1.0 / V)
    G = damping * M + (1 - damping) / V
    pr = np.full(V, 1.0 / V)
    for _ in range(iterations):
        pr = G @ pr
    return pr


def test_pagerank_matches_dense_power_iteration():
    rng = np.random.default_rng(9)
    for n in (1, 3, 20, 200):
        for _ in range(5):
            s = rng.integers(-8, 8, n).astype(np.int32)
            d = rng.integers(-8, 8, n).astype(np.int32)
            g = oracle.table_to_graph(s, d)
            for iters in (0, 1, 10, 30):
                got = oracle.pagerank(g, 0.85, iters)
                want = dense_pagerank(s, d, 0.85, iters)
                assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
    for t in (pins.load_golden(p) for p in pins.golden_files()):
        if len(t["src"]):
            g = oracle.table_to_graph(t["src"], t["dst"])
            assert np.allclose(oracle.pagerank(g), dense_pagerank(t["src"], t["dst"]), rtol=1e-12)


def test_pagerank_closed_forms_and_conservation():
    # a directed cycle stays uniform; one self-loop holds all the rank
    n = 7
    s = np.arange(n, dtype=np.int32)
    g = oracle.table_to_graph(s, (s + 1) % n)
    assert np.allclose(oracle.pagerank(g, 0.85, 10), 1.0 / n, rtol=0, atol=1e-15)
    g = oracle.table_to_graph(np.array([4], np.int32), np.array([4], np.int32))
    assert np.allclose(oracle.pagerank(g), [1.0])
    # two nodes a -> b: b is dangling; after one step
    # PR(a) = (1-d)/2 + d*(0.5/2), PR(b) = (1-d)/2 + d*(0.5 + 0.5/2)
    g = oracle.table_to_graph(np.array([1], np.int32), np.array([2], np.int32))
    d = 0.85
    assert np.allclose(oracle.pagerank(g, d, 1), [(1 - d) / 2 + d * 0.25, (1 - d) / 2 + d * 0.75])
    # the total rank stays 1
    s, dd = tg.make_table(tg.SPECS["lj"].scaled(20_000), seed=3)
    g = oracle.table_to_graph(s.numpy(), dd.numpy())
    assert abs(oracle.pagerank(g).sum() - 1.0) < 1e-12


def test_pagerank_star_two_state_recurrence():
    # k leaves each pointing at one hub (the hub has no out-edges): by symmetry
    # every leaf has the same rank, so ten steps reduce to a recurrence on two
    # numbers, evaluated here in exact rational arithmetic
    from fractions import Fraction as F
    k, d = 9, F(85, 100)
    V = k + 1
    leaf, hub = F(1, V), F(1, V)
    for _ in range(10):
        leaf, hub = (1 - d) / V + d * hub / V, (1 - d) / V + d * (k * leaf + hub / V)
    s = np.arange(100, 100 + k, dtype=np.int32)  # leaves 100.., hub 5 sorts first
    g = oracle.table_to_graph(s, np.full(k, 5, np.int32))
    got = oracle.pagerank(g, 0.85, 10)
    assert got[0] == pytest.approx(float(hub), rel=1e-14)
    assert np.allclose(got[1:], float(leaf), rtol=1e-14, atol=0)


def test_pagerank_pins_catch_dropped_dangling_mass():
    g = oracle.table_to_graph(np.array([1, 1, 3], np.int32), np.array([2, 3, 1], np.int32))
    bad = oracle.pagerank(g, drop_dangling=True)
    assert abs(bad.sum() - 1.0) > 1e-3
    assert not np.allclose(bad, dense_pagerank([1, 1, 3], [2, 3, 1]), rtol=1e-6)


# ------------------------------------------------- undirected + triangles ---
def dense_triangles(src, dst) -> int:
    """trace(A^3) / 6 with the symmetric 0/1 adjacency matrix of the distinct
    unordered pairs, loops removed: a route independent of the CSR."""
    ids = sorted(set(int(x) for x in src) | set(int(x) for x in dst))
    idx = {x: i for i, x in enumerate(ids)}
    A = np.zeros((len(ids), len(ids)), dtype=np.int64)
    for a, b in zip(src, dst):
        if a != b:
            A[idx[int(a)], idx[int(b)]] = A[idx[int(b)], idx[int(a)]] = 1
    return int(np.trace(A @ A @ A)) // 6


def test_undirected_graph_is_symmetric_set_of_pairs():
    rng = np.random.default_rng(12)
    for n in (0, 1, 5, 60):
        s = rng.integers(-6, 6, n).astype(np.int32)
        d = rng.integers(-6, 6, n).astype(np.int32)
        g = oracle.undirected_graph(s, d)
        ids = g["node_ids"]
        adj = {int(ids[r]): set(int(ids[k]) for k in g["out_nbr"][g["out_off"][r]:g["out_off"][r + 1]])
               for r in range(g["num_nodes"])}
        want = {}
        for a, b in zip(s.tolist(), d.tolist()):
            want.setdefault(a, set()).add(b)
            want.setdefault(b, set()).add(a)
        assert adj == want
        for d_ in ("off", "nbr"):
            assert np.array_equal(g[f"out_{d_}"], g[f"in_{d_}"])


def test_triangles_match_dense_count():
    rng = np.random.default_rng(13)
    for n in (0, 3, 20, 120, 400):
        for _ in range(4):
            s = rng.integers(0, 25, n).astype(np.int32)
            d = rng.integers(0, 25, n).astype(np.int32)
            assert oracle.count_triangles(oracle.undirected_graph(s, d)) == dense_triangles(s, d)


def test_triangles_closed_forms():
    import itertools
    from math import comb
    for n in (3, 4, 7, 12):  # complete graph
        p = list(itertools.combinations(range(n), 2))
        g = oracle.undirected_graph([a for a, _ in p], [b for _, b in p])
        assert oracle.count_triangles(g) == comb(n, 3)
    for n in (3, 4, 9):  # cycle
        v = np.arange(n, dtype=np.int32)
        assert oracle.count_triangles(oracle.undirected_graph(v, (v + 1) % n)) == (1 if n == 3 else 0)
    for n in (4, 8):  # wheel: a hub joined to every node of an n-cycle
        v = np.arange(n, dtype=np.int32)
        s = np.concatenate([v, np.full(n, 100, np.int32)])
        d = np.concatenate([(v + 1) % n, v])
        assert oracle.count_triangles(oracle.undirected_graph(s, d)) == n
    # loops, duplicates and reversed rows change nothing
    s = np.array([1, 2, 3, 1, 2, 3, 3, 2], np.int32)
    d = np.array([2, 3, 1, 1, 1, 3, 2, 2], np.int32)
    assert oracle.count_triangles(oracle.undirected_graph(s, d)) == 1
    # a complete bipartite graph has none; k disjoint triangles have k; a
    # complete graph minus one edge has C(n, 3) - (n - 2)
    a, b = np.meshgrid(np.arange(6, dtype=np.int32), np.arange(10, 17, dtype=np.int32))
    assert oracle.count_triangles(oracle.undirected_graph(a.ravel(), b.ravel())) == 0
    t = np.arange(0, 300, 3, dtype=np.int32)
    s = np.concatenate([t, t + 1, t + 2])
    d = np.concatenate([t + 1, t + 2, t])
    assert oracle.count_triangles(oracle.undirected_graph(s, d)) == 100
    n = 9
    p = [q for q in itertools.combinations(range(n), 2) if q != (2, 5)]
    g = oracle.undirected_graph([x for x, _ in p], [y for _, y in p])
    assert oracle.count_triangles(g) == comb(n, 3) - (n - 2)


def test_triangle_pins_catch_planted_mistake():
    p = [(0, 1), (1, 2), (0, 2), (2, 3)]
    g = oracle.undirected_graph([a for a, _ in p], [b for _, b in p])
    assert oracle.count_triangles(g, mutant=9) != dense_triangles([a for a, _ in p], [b for _, b in p])


# ----------------------------------------------------------- select / join ---
def test_select_is_the_ordered_filter():
    import operator
    ops = {"<": operator.lt, "<=": operator.le, "==": operator.eq, "!=": operator.ne,
           ">=": operator.ge, ">": operator.gt}
    rng = np.random.default_rng(14)
    for n in (0, 1, 7, 300):
        s = rng.integers(-5, 5, n).astype(np.int32)
        d = rng.integers(-5, 5, n).astype(np.int32)
        for col in (0, 1):
            for op, fn in ops.items():
                for v in (-6, -1, 0, 3, 6):
                    got = oracle.table_select(s, d, col, op, v)
                    want = [(a, b) for a, b in zip(s.tolist(), d.tolist()) if fn((b if col else a), v)]
                    assert list(zip(got[0].tolist(), got[1].tolist())) == want
        # complementary comparisons split the table
        for v in (-2, 0, 4):
            assert oracle.table_select(s, d, 0, "<", v)[0].size + \
                oracle.table_select(s, d, 0, ">=", v)[0].size == n


def test_join_is_the_nested_loop():
    rng = np.random.default_rng(15)
    for n in (0, 1, 9, 200):
        s = rng.integers(-4, 4, n).astype(np.int32)
        d = rng.integers(-4, 4, n).astype(np.int32)
        for nk in (0, 1, 5, 30):
            keys = rng.integers(-5, 5, nk).astype(np.int32)
            for col in (0, 1):
                got = oracle.table_join(s, d, col, keys)
                want = [(a, b) for a, b in zip(s.tolist(), d.tolist())
                        for k in keys.tolist() if (b if col else a) == k]
                assert list(zip(got[0].tolist(), got[1].tolist())) == want
    # every key once: the join keeps the whole table
    s = rng.integers(0, 50, 400).astype(np.int32)
    d = rng.integers(0, 50, 400).astype(np.int32)
    out = oracle.table_join(s, d, 0, np.unique(s))
    assert np.array_equal(out[0], s) and np.array_equal(out[1], d)
