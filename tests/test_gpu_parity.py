"""CUDA path vs the oracle, element by element, through the C ABI.

Integer work: the bar is bit-exact equality of all five arrays plus V and E.
Sizes span one partial tile up to many 4096-key tiles with ragged tails; the
full-size workloads (69M and 1.47B rows) are checked on sampled nodes against
the oracle's scan and on whole-table properties.
"""
import numpy as np
import pytest
import torch

import gpu_checks
import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def gpu_convert(src, dst) -> dict:
    s = torch.as_tensor(np.ascontiguousarray(src, np.int32)).cuda()
    d = torch.as_tensor(np.ascontiguousarray(dst, np.int32)).cuda()
    g = ringo.ringo_table_to_graph(s, d)
    try:
        return g.copy_to_host()
    finally:
        g.free()


def compare_with_oracle(src, dst, what=""):
    src = np.asarray(src, np.int32)
    dst = np.asarray(dst, np.int32)
    pins.assert_same_graph(gpu_convert(src, dst), oracle.table_to_graph(src, dst), what)


def test_golden_tables():
    pins.check_golden(gpu_convert)


def test_brute_force_exhaustive():
    pins.check_brute_force_exhaustive(gpu_convert, alphabet=(-1, 0, 1, 2), max_rows=3)


def test_brute_force_random_extreme_ids():
    pins.check_brute_force_random(gpu_convert, trials=300)


def test_special_cases():
    pins.check_special_cases(gpu_convert)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 511, 4095, 4096, 4097, 8191, 12289, 65537,
                               100_003])
def test_ragged_sizes(n):
    s, d = tg.signed_table(n, max(2, n // 7), seed=n)
    compare_with_oracle(s.numpy(), d.numpy(), f"signed n={n}")


@pytest.mark.parametrize("spec", ["tiny", "lj", "twitter"])
def test_shapes_scaled(spec):
    sp = tg.SPECS[spec].scaled(1_500_017)
    s, d = tg.make_table(sp, seed=2)
    compare_with_oracle(s.numpy(), d.numpy(), sp.name)


def test_tiny_config_full():
    s, d = tg.make_table("tiny", seed=1)
    compare_with_oracle(s.numpy(), d.numpy(), "tiny 1M")


def test_generator_same_on_cpu_and_gpu():
    sp = tg.SPECS["twitter"].scaled(300_000)
    sc, dc = tg.make_table(sp, seed=4, device="cpu")
    sg, dg = tg.make_table(sp, seed=4, device="cuda")
    assert torch.equal(sc, sg.cpu()) and torch.equal(dc, dg.cpu())


def test_small_id_range_skips_passes():
    # IDs in [0, 200): the top digits never vary, so radix passes are skipped
    rng = np.random.default_rng(5)
    s = rng.integers(0, 200, 50_000).astype(np.int32)
    d = rng.integers(0, 200, 50_000).astype(np.int32)
    compare_with_oracle(s, d, "small range")
    g = ringo.ringo_table_to_graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    info = g.info()
    assert info["out_sort_passes"] == 2 and info["in_sort_passes"] == 1


def test_all_rows_identical_and_single_row():
    compare_with_oracle(np.full(10_000, 7, np.int32), np.full(10_000, -3, np.int32), "identical")
    compare_with_oracle(np.array([5], np.int32), np.array([5], np.int32), "one loop")


def test_empty_table():
    g = ringo.ringo_table_to_graph(torch.empty(0, dtype=torch.int32, device="cuda"),
                                   torch.empty(0, dtype=torch.int32, device="cuda"))
    a = g.copy_to_host()
    assert a["num_nodes"] == 0 and a["num_edges"] == 0
    assert a["out_off"].tolist() == [0] and a["in_off"].tolist() == [0]


def test_row_order_and_duplicates():
    s, d = tg.signed_table(30_000, 4_000, seed=12)
    pins.check_row_order_and_duplicates(gpu_convert, s.numpy(), d.numpy())


def test_unaligned_columns_and_host_entry():
    s, d = tg.signed_table(20_001, 3_000, seed=13)
    want = oracle.table_to_graph(s.numpy()[1:], d.numpy()[1:])
    sg, dg = s.cuda(), d.cuda()
    g = ringo.ringo_table_to_graph(sg[1:], dg[1:])  # 4-byte offset: not 16-byte aligned
    pins.assert_same_graph(g.copy_to_host(), want, "unaligned")
    h = ringo.ringo_table_to_graph_host(s.numpy()[1:], d.numpy()[1:])
    pins.assert_same_graph(h.copy_to_host(), want, "host entry")
    hp = ringo.ringo_table_to_graph_host(s[1:].clone().pin_memory(), d[1:].clone().pin_memory())
    pins.assert_same_graph(hp.copy_to_host(), want, "pinned host entry")


@pytest.mark.parametrize("n", [0, 1, 4097, 200_003])
def test_host_io_entry(n):
    """Host columns in, host arrays out: the out-CSR comes back on a second
    stream while the in-CSR is built; the result equals the oracle's."""
    s, d = tg.signed_table(n, max(2, n // 5), seed=17) if n else (
        torch.empty(0, dtype=torch.int32), torch.empty(0, dtype=torch.int32))
    want = oracle.table_to_graph(s.numpy(), d.numpy())
    got = ringo.ringo_table_to_graph_host_io(s.pin_memory() if n else s,
                                             d.pin_memory() if n else d)
    pins.assert_same_graph({k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in got.items()},
                           want, f"host io, {n} rows")
    if n:
        # pageable numpy columns and caller-owned (pageable) outputs
        out = {"node_ids": torch.empty(2 * n, dtype=torch.int32),
               "out_off": torch.empty(2 * n + 1, dtype=torch.int64),
               "out_nbr": torch.empty(n, dtype=torch.int32),
               "in_off": torch.empty(2 * n + 1, dtype=torch.int64),
               "in_nbr": torch.empty(n, dtype=torch.int32)}
        got2 = ringo.ringo_table_to_graph_host_io(s.numpy(), d.numpy(), out=out)
        pins.assert_same_graph({k: (v.numpy() if hasattr(v, "numpy") else v)
                                for k, v in got2.items()}, want, f"host io pageable, {n} rows")


def test_host_io_capacity_errors():
    s, d = tg.signed_table(5000, 1000, seed=19)
    want = oracle.table_to_graph(s.numpy(), d.numpy())
    V = int(want["num_nodes"])
    small = {"node_ids": torch.empty(V - 1, dtype=torch.int32),
             "out_off": torch.empty(V, dtype=torch.int64),
             "out_nbr": torch.empty(5000, dtype=torch.int32),
             "in_off": torch.empty(V, dtype=torch.int64),
             "in_nbr": torch.empty(5000, dtype=torch.int32)}
    with pytest.raises(ringo.RingoError) as ei:
        ringo.ringo_table_to_graph_host_io(s, d, out=small)
    assert ei.value.status == ringo.RINGO_ERANGE
    exact = dict(small, node_ids=torch.empty(V, dtype=torch.int32),
                 out_off=torch.empty(V + 1, dtype=torch.int64),
                 in_off=torch.empty(V + 1, dtype=torch.int64))
    got = ringo.ringo_table_to_graph_host_io(s, d, out=exact)
    pins.assert_same_graph({k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in got.items()},
                           want, "exact capacity")


def test_degrees_and_topk():
    s, d = tg.make_table(tg.SPECS["twitter"].scaled(400_000), seed=6)
    want = oracle.table_to_graph(s.numpy(), d.numpy())
    g = ringo.ringo_table_to_graph(s.cuda(), d.cuda())
    ids = want["node_ids"]
    q = np.r_[ids[::97], np.int32(-5), np.int32(2**31 - 1)]
    for di, name in ((0, "out"), (1, "in")):
        deg = np.diff(want[f"{name}_off"])
        r = np.searchsorted(ids, q)
        hit = (r < ids.size) & (ids[np.minimum(r, ids.size - 1)] == q)
        exp = np.where(hit, deg[np.minimum(r, ids.size - 1)], -1)
        got = g.degrees(di, torch.from_numpy(q)).cpu().numpy()
        assert np.array_equal(got, exp)
        assert g.degree(di, int(ids[5])) == int(deg[5])
        with pytest.raises(ringo.RingoError) as e:
            g.degree(di, -5 if -5 not in ids else 2**31 - 2)
        assert e.value.status == ringo.RINGO_ENOTFOUND
        for k in (1, 100, 4096):
            tid, tdeg = g.degree_topk(di, k)
            order = np.lexsort((ids, -deg))[:k]
            assert np.array_equal(tid, ids[order]) and np.array_equal(tdeg, deg[order])


def _full_size(spec: str, seed: int, n_random: int):
    src, dst = tg.make_table(spec, seed=seed, device="cuda")
    g = ringo.ringo_table_to_graph(src, dst)
    a = gpu_checks.graph_arrays(g)
    gpu_checks.check_properties(a, src, dst)
    src_h, dst_h = src.cpu().numpy(), dst.cpu().numpy()
    ids = a["node_ids"].cpu().numpy()
    sample = gpu_checks.pick_samples(src_h, dst_h, ids, a, n_random=n_random)
    gpu_checks.check_samples(a, src_h, dst_h, sample)
    e, v = g.num_edges, g.num_nodes
    g.free()
    return e, v


def test_lj_full_size_sampled():
    e, v = _full_size("lj", 1, 300)
    assert 6.5e7 < e < 6.9e7 and 4.5e6 < v <= 4.85e6


@pytest.mark.slow
def test_twitter_full_size_sampled():
    e, v = _full_size("twitter", 1, 100)
    assert 1.4e9 < e < 1.47e9 and 3.5e7 < v <= 4.17e7


@pytest.mark.parametrize("src_only", [0, 1, 31, 32, 33, 255, 256, 257, 2000])
def test_out_remap_step_list_threshold(src_only):
    """The out-direction remap uses a short list of the map's steps when at
    most 256 nodes are not destinations, else block tables: both paths, and
    the boundary, against the oracle."""
    rng = np.random.default_rng(100 + src_only)
    dst_ids = np.arange(0, 3 * 60_000, 3, dtype=np.int64)          # 60K destinations
    extra = rng.choice(np.arange(1, 3 * 60_000, 3), src_only, replace=False)  # between them
    n = 250_000
    src = rng.choice(np.concatenate([dst_ids, extra]), n)
    dst = rng.choice(dst_ids, n)
    # every destination and every extra source occurs
    src[:src_only] = extra
    dst[:dst_ids.size] = dst_ids
    s, d = src.astype(np.int32), dst.astype(np.int32)
    want = oracle.table_to_graph(s, d)
    g = ringo.ringo_table_to_graph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    inf = g.info()
    assert inf["num_nodes"] - inf["num_dst_nodes"] == src_only
    pins.assert_same_graph(g.copy_to_host(), want, f"{src_only} source-only nodes")
    g.free()


@pytest.mark.parametrize("gap", [0, 1, 30, 31, 32, 33, 5000])
def test_in_offsets_across_nodes_without_in_edges(gap):
    """Nodes that are only sources have empty in-lists, so their in-offset is
    the next destination's: runs of `gap` such nodes before the first
    destination, between destinations and after the last, across the length
    where the destination-run kernel stops writing a run itself and records
    it for the range fill, against the oracle."""
    rng = np.random.default_rng(300 + gap)
    ndst = 40
    ids = (np.arange((ndst + 1) * (gap + 1), dtype=np.int64) * 7 - 900).astype(np.int32)
    is_dst = np.zeros(ids.size, bool)
    is_dst[gap::gap + 1][:ndst] = True
    dsts, only_src = ids[is_dst], ids[~is_dst]
    # every source-only node points at some destination; every destination
    # has an in-edge (from the next destination, so that destinations are
    # sources too for half of them)
    src = [only_src, dsts]
    dst = [rng.choice(dsts, only_src.size) if only_src.size else only_src, np.roll(dsts, 1)]
    src = np.concatenate(src).astype(np.int32)
    dst = np.concatenate(dst).astype(np.int32)
    p = rng.permutation(src.size)
    src, dst = src[p], dst[p]
    g = ringo.ringo_table_to_graph(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    got = g.copy_to_host()
    g.free()
    pins.assert_same_graph(got, oracle.table_to_graph(src, dst), f"gap {gap}")
