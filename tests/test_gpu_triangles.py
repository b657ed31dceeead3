"""Undirected conversion and triangle counting through the C ABI, against the
oracle: the undirected graph bit for bit, the triangle count exactly."""
import itertools
from math import comb

import numpy as np
import pytest
import torch

import gpu_checks
import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def gpu_undirected(src, dst):
    s = torch.as_tensor(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.as_tensor(np.ascontiguousarray(dst, np.int32)).cuda()
    g = ringo.ringo_table_to_undirected_graph(s, d)
    try:
        return g.copy_to_host(), g.count_triangles()
    finally:
        g.free()


def check(src, dst, what=""):
    got, tri = gpu_undirected(src, dst)
    want = oracle.undirected_graph(src, dst)
    pins.assert_same_graph(got, want, what)
    assert tri == oracle.count_triangles(want), what


def test_golden_tables():
    for path in pins.golden_files():
        t = pins.load_golden(path)
        check(t["src"], t["dst"], path)


@pytest.mark.parametrize("n", [1, 2, 3, 4097, 100_003])
def test_signed_tables(n):
    s, d = tg.signed_table(n, max(3, n // 9), seed=n + 1)
    check(s.numpy(), d.numpy(), f"n={n}")


@pytest.mark.parametrize("spec", ["tiny", "lj", "twitter"])
def test_shapes_scaled(spec):
    sp = tg.SPECS[spec].scaled(600_011)
    s, d = tg.make_table(sp, seed=8)
    check(s.numpy(), d.numpy(), sp.name)


def test_closed_forms():
    for n in (3, 5, 40, 200):
        p = list(itertools.combinations(range(n), 2))
        _, tri = gpu_undirected(np.array([a for a, _ in p]), np.array([b for _, b in p]))
        assert tri == comb(n, 3)
    v = np.arange(1000, dtype=np.int32)
    _, tri = gpu_undirected(v, (v + 1) % 1000)
    assert tri == 0


def test_large_clique():
    # a 1100-clique: oriented lists of every length from 0 to 1099, and
    # C(1100, 3) = 221,228,700 triangles in one 64-bit total
    n = 1100
    a, b = np.triu_indices(n, 1)
    _, tri = gpu_undirected(a.astype(np.int32) * 3, b.astype(np.int32) * 3)
    assert tri == comb(n, 3)


def test_hub_and_clique():
    # a hub joined to 50K nodes, and a 60-clique among some of them: the hub
    # is ordered last, the clique's triangles are found from its members
    hub = np.full(50_000, -9, np.int32)
    leaves = np.arange(50_000, dtype=np.int32) * 7
    p = list(itertools.combinations(range(60), 2))
    cs = np.array([leaves[a] for a, _ in p], np.int32)
    cd = np.array([leaves[b] for _, b in p], np.int32)
    check(np.concatenate([hub, cs]), np.concatenate([leaves, cd]), "hub+clique")


def test_lj_full_size_invariance():
    src, dst = tg.make_table("lj", seed=2, device="cuda")
    g = ringo.ringo_table_to_undirected_graph(src, dst)
    t1 = g.count_triangles()
    assert t1 > 0 and g.count_triangles() == t1
    off, nbr = g.csr(ringo.RINGO_OUT)
    off2, nbr2 = g.csr(ringo.RINGO_IN)
    assert torch.equal(off, off2) and torch.equal(nbr, nbr2)
    g.free()
    # the same edges in another row order and direction
    perm = torch.randperm(src.numel(), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    flip = torch.rand(src.numel(), device="cuda") < 0.5
    s2 = torch.where(flip, dst[perm], src[perm]).contiguous()
    d2 = torch.where(flip, src[perm], dst[perm]).contiguous()
    g2 = ringo.ringo_table_to_undirected_graph(s2, d2)
    assert g2.count_triangles() == t1
    g2.free()


def test_reciprocal_edges_and_hub_splits():
    """Mutual edges (the same pair in both directions, and repeated) are one
    undirected edge; hubs whose lists span many merge blocks are split inside
    the node, at ties between the two lists too."""
    rng = np.random.default_rng(21)
    a = rng.integers(-50_000, 50_000, 300_000).astype(np.int32)
    b = rng.integers(-50_000, 50_000, 300_000).astype(np.int32)
    half = rng.random(300_000) < 0.5
    src = np.concatenate([a, b[half], a[:1000]])
    dst = np.concatenate([b, a[half], b[:1000]])
    check(src, dst, "reciprocal")
    leaves = np.arange(0, 120_000, dtype=np.int32) * 3 + 1
    hub_out = np.full(leaves.size, -5, np.int32)
    evens = leaves[::2]
    src = np.concatenate([hub_out, evens, np.full(7_000, 2, np.int32), evens[:7_000]])
    dst = np.concatenate([leaves, np.full(evens.size, -5, np.int32), evens[:7_000],
                          np.full(7_000, 2, np.int32)])
    check(src, dst, "hubs")


@pytest.mark.slow
def test_twitter_full_size_undirected():
    """The Twitter-shaped table (1.47B rows, above 2^30) in undirected form,
    checked at full size: the directed graph's invariants, every undirected
    list the union of the node's out- and in-lists, oracle lists of sampled
    nodes, and a positive triangle count that a second run repeats."""
    src, dst = tg.make_table("twitter", seed=1, device="cuda")
    gd = ringo.ringo_table_to_graph(src, dst)
    d = gpu_checks.graph_arrays(gd)
    gpu_checks.check_properties(d, src, dst)
    g = ringo.ringo_table_to_undirected_graph(src, dst)
    u = gpu_checks.graph_arrays(g)
    gpu_checks.check_undirected(u, d)
    del d
    gd.free()
    src_h, dst_h = src.cpu().numpy(), dst.cpu().numpy()
    ids = u["node_ids"].cpu().numpy()
    sample = gpu_checks.pick_samples(src_h, dst_h, ids, u, n_random=60)
    gpu_checks.check_undirected_samples(u, src_h, dst_h, sample)
    del u, src_h, dst_h
    tri = g.count_triangles()
    assert tri > 0 and g.count_triangles() == tri
    g.free()
