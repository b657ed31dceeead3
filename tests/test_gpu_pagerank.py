"""PageRank on the built graph (the paper's second workload, ten iterations)
through the C ABI, against the oracle's fp64 power iteration.

Tolerance: the GPU forms each node's sum over its in-edges in another order
than the oracle (8-edge runs, a scan over a tile's threads, then the shares of
the 2048-edge tiles a node spans, in tile order), and the
dangling mass by a tree of block sums.  Reordering an fp64 sum of k positive
terms changes it by at most (k - 1) * 2^-53 relative; with in-degrees below
3e6 and the dangling sum over at most 4.2e7 nodes that is below 5e-9 per
step, and steps damp earlier errors by d <= 1, so 10 steps stay within
rtol = 1e-7 at the largest sizes here and far inside it at small ones.
"""
import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu

RTOL = 1e-7


def gpu_pagerank(src, dst, damping=0.85, iterations=10):
    s = torch.as_tensor(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.as_tensor(np.ascontiguousarray(dst, np.int32)).cuda()
    g = ringo.ringo_table_to_graph(s, d)
    try:
        pr = g.pagerank(damping, iterations)
        torch.cuda.synchronize()
        return pr.cpu().numpy(), g.copy_to_host()
    finally:
        g.free()


def check(src, dst, damping=0.85, iterations=10, what=""):
    got, g = gpu_pagerank(src, dst, damping, iterations)
    want = oracle.pagerank(oracle.table_to_graph(src, dst), damping, iterations)
    assert got.shape == want.shape, what
    assert np.allclose(got, want, rtol=RTOL, atol=0), \
        f"{what}: max rel err {np.max(np.abs(got - want) / want) if want.size else 0}"


def test_golden_tables():
    for path in pins.golden_files():
        t = pins.load_golden(path)
        check(t["src"], t["dst"], what=path)


@pytest.mark.parametrize("damping,iterations", [(0.85, 0), (0.85, 1), (0.85, 10), (0.5, 10),
                                                (1.0, 10), (0.0, 3)])
def test_damping_and_iterations(damping, iterations):
    s, d = tg.signed_table(20_011, 3_000, seed=2)
    check(s.numpy(), d.numpy(), damping, iterations, f"d={damping} it={iterations}")


@pytest.mark.parametrize("n", [1, 2, 4097, 100_003])
def test_ragged_sizes(n):
    s, d = tg.signed_table(n, max(2, n // 7), seed=n)
    check(s.numpy(), d.numpy(), what=f"n={n}")


@pytest.mark.parametrize("spec", ["tiny", "lj", "twitter"])
def test_shapes_scaled(spec):
    sp = tg.SPECS[spec].scaled(1_500_017)
    s, d = tg.make_table(sp, seed=7)
    check(s.numpy(), d.numpy(), what=sp.name)


def test_hub_node_and_dangling_nodes():
    # 300K edges into one node (spans many edge tiles), and many nodes with
    # no out-edges
    n = 300_000
    s = np.arange(n, dtype=np.int32) + 10
    d = np.full(n, 3, np.int32)
    s = np.concatenate([s, np.array([3, 3], np.int32)])
    d = np.concatenate([d, np.array([5, 7], np.int32)])
    check(s, d, what="hub")


def test_lj_full_size():
    src, dst = tg.make_table("lj", seed=1, device="cuda")
    g = ringo.ringo_table_to_graph(src, dst)
    del src, dst
    pr = g.pagerank(0.85, 10).cpu().numpy()
    h = g.copy_to_host()
    g.free()
    want = oracle.pagerank(h, 0.85, 10)
    assert np.allclose(pr, want, rtol=RTOL, atol=0)
    assert abs(pr.sum() - 1.0) < 1e-9


def test_argument_errors():
    g = ringo.ringo_table_to_graph(torch.tensor([1], dtype=torch.int32, device="cuda"),
                                   torch.tensor([2], dtype=torch.int32, device="cuda"))
    for damping, it in ((1.5, 10), (-0.1, 10), (0.85, -1)):
        with pytest.raises(ringo.RingoError) as e:
            g.pagerank(damping, it)
        assert e.value.status == ringo.RINGO_EINVAL
    g.free()


def test_same_bits_on_every_run():
    # each node's sum is formed in a fixed order: two runs agree bit for bit,
    # also with a hub node cut across many edge tiles
    n = 40_000
    s = np.concatenate([np.arange(n, dtype=np.int32) + 100,
                        np.random.default_rng(1).integers(0, 5000, 200_000).astype(np.int32)])
    d = np.concatenate([np.full(n, 7, np.int32),
                        np.random.default_rng(2).integers(0, 5000, 200_000).astype(np.int32)])
    g = ringo.ringo_table_to_graph(torch.as_tensor(s).cuda(), torch.as_tensor(d).cuda())
    a = g.pagerank(0.85, 10).clone()
    b = g.pagerank(0.85, 10)
    assert torch.equal(a, b)
    g.free()
