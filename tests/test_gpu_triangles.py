"""Undirected conversion and triangle counting through the C ABI, against the
oracle: the undirected graph bit for bit, the triangle count exactly."""
import itertools
from math import comb

import numpy as np
import pytest
import torch

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
