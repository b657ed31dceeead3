"""The tuner's knobs and its cache.

Every radix pass variant the tuner can choose (peer detection by lane masks,
per-bit ballots or a warp match; L2 prefetch 0, 1 or 2 waves ahead; 8- or
9-bit in-direction digits) must give the same graph as the oracle, bit for
bit, on tables across tile boundaries, signed IDs, skewed digits, more than
2^18 distinct destinations (three active 9-bit passes) and a batch; a tuned
choice is recorded per size class, written to the JSON cache and reused by
a later process without tuning."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
VARIANTS = ([{"rank_method": r, "prefetch_waves": w, "in_digit_bits": 8}
             for r in (0, 1, 2) for w in (0, 1, 2)]
            + [{"rank_method": r, "prefetch_waves": 1, "in_digit_bits": 9} for r in (0, 1, 2)])


def _vid(o):
    return f"rank{o['rank_method']}-pf{o['prefetch_waves']}-in{o['in_digit_bits']}"


@pytest.fixture
def forced():
    yield lambda o: ringo.ringo_sort_opts_force(o)
    ringo.ringo_sort_opts_force(None)


def _tables():
    out = []
    for n in (1, 4095, 4097, 65537):
        out.append(tg.signed_table(n, max(2, n // 7), seed=60 + n % 97))
    out.append(tg.make_table(tg.SPECS["tiny"].scaled(300_000), seed=61))  # Zipf(1.1) sources
    out.append(tg.make_table(tg.SPECS["lj"].scaled(400_000), seed=62))
    # every key shares its low digits: one digit value per pass for most keys
    s = (torch.arange(200_000, dtype=torch.int64) % 5 * 256).to(torch.int32)
    d = (torch.arange(200_000, dtype=torch.int64) % 3 * 65536).to(torch.int32)
    out.append((s, d))
    # distinct destinations above 2^18: three 9-bit (four 8-bit) in-passes
    g = torch.Generator().manual_seed(67)
    s = torch.randint(0, 5_000, (700_000,), generator=g, dtype=torch.int32)
    d = torch.randint(-(1 << 31), (1 << 31) - 1, (700_000,), generator=g, dtype=torch.int32)
    out.append((s, d))
    return out


@pytest.mark.parametrize("opts", VARIANTS, ids=_vid)
def test_every_pass_variant_matches_the_oracle(opts, forced):
    forced(opts)
    for s, d in _tables():
        want = oracle.table_to_graph(s.numpy(), d.numpy())
        g = ringo.ringo_table_to_graph(s.cuda(), d.cuda())
        got = g.copy_to_host()
        g.free()
        pins.assert_same_graph(got, want, f"{opts}, {s.numel()} rows")


@pytest.mark.parametrize("rank", (0, 1, 2))
@pytest.mark.parametrize("bits", (8, 9))
def test_batch_with_each_rank_method(rank, bits, forced):
    forced({"rank_method": rank, "prefetch_waves": 1, "in_digit_bits": bits})
    spec = tg.BaseSpec(rows=400_000, nodes=50_000, tags=300)
    cols = tg.make_base_table(spec, seed=63)
    preds = tg.make_predicates(spec, 40, 50, 40_000, seed=63)
    base = ringo.BaseTable(*(c.cuda() for c in cols))
    src, dst, ts, tag = (c.numpy() for c in cols)
    try:
        bt = base.convert_batch(preds)
        for i, (tags, t0, t1) in enumerate(preds):
            m = np.isin(tag, np.asarray(tags, np.int32)) & (ts >= t0) & (ts < t1)
            pins.assert_same_graph(bt.copy_to_host(i), oracle.table_to_graph(src[m], dst[m]),
                                   f"rank {rank}, {bits}-bit, selection {i}")
        bt.free()
    finally:
        base.free()


def test_tuned_choice_is_recorded_cached_and_reused(tmp_path):
    cache = str(tmp_path / "ringo_tune.json")
    ringo.ringo_tune_set_cache(cache)
    try:
        src, dst = tg.make_table(tg.SPECS["lj"].scaled(1_500_000), seed=64, device="cuda")
        best, ms = ringo.ringo_tune_table(src, dst)
        assert ms > 0 and best["rank_method"] in (0, 1, 2) and 0 <= best["prefetch_waves"] <= 2
        assert best["in_digit_bits"] in (8, 9)
        found, got = ringo.ringo_tune_lookup(0, src.numel())
        assert found and got["rank_method"] == best["rank_method"]
        assert got["prefetch_waves"] == best["prefetch_waves"]
        assert got["in_digit_bits"] == best["in_digit_bits"]
        # a table of the same size class uses the choice; the result is exact
        s2, d2 = tg.make_table(tg.SPECS["lj"].scaled(1_100_000), seed=65, device="cuda")
        g = ringo.ringo_table_to_graph(s2, d2)
        pins.assert_same_graph(g.copy_to_host(),
                               oracle.table_to_graph(s2.cpu().numpy(), d2.cpu().numpy()),
                               "tuned class")
        g.free()
        entries = json.load(open(cache))["entries"]
        mine = [e for e in entries if e["kind"] == 0 and e["size_class"] == src.numel().bit_length() - 1]
        assert len(mine) == 1 and mine[0]["rank_method"] == best["rank_method"]
        assert mine[0]["in_digit_bits"] == best["in_digit_bits"]
        assert mine[0]["out_passes"] >= 1
        # a fresh process reads the file and finds the choice without tuning
        code = ("import sys; sys.path.insert(0, %r); from paper_1503_07881_gb300 import ringo; "
                "ringo.ringo_tune_set_cache(%r); f, o = ringo.ringo_tune_lookup(0, %d); "
                "print(int(f), o['rank_method'], o['prefetch_waves'], o['in_digit_bits'])"
                % (ROOT, cache, src.numel()))
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0, out.stderr
        f, r, w, b = map(int, out.stdout.split()[-4:])
        assert (f, r, w, b) == (1, best["rank_method"], best["prefetch_waves"],
                                best["in_digit_bits"])
    finally:
        ringo.ringo_tune_set_cache(None)


def test_batch_autotune_records_a_batch_choice(tmp_path):
    cache = str(tmp_path / "ringo_tune_batch.json")
    ringo.ringo_tune_set_cache(cache)
    spec = tg.BaseSpec(rows=600_000, nodes=80_000, tags=300)
    cols = tg.make_base_table(spec, seed=66)
    preds = tg.make_predicates(spec, 32, 1_000, 60_000, seed=66)
    base = ringo.BaseTable(*(c.cuda() for c in cols))
    try:
        wave, ms = base.autotune(preds)
        assert wave > 0 and ms > 0
        counts = base.select_count(preds)
        found, o = ringo.ringo_tune_lookup(1, int(counts.sum()) // len(preds))
        assert found and o["wave_rows"] == wave
        kinds = {e["kind"] for e in json.load(open(cache))["entries"]}
        assert 1 in kinds
    finally:
        ringo.ringo_tune_set_cache(None)
        base.free()
