"""Host logic of the synthetic base tables and predicates (no GPU)."""
import numpy as np

from paper_1503_07881_gb300 import tablegen as tg


def expected_rows(spec, pred):
    tags, t0, t1 = pred
    share = tg.tag_row_counts(spec)[tags].sum()
    lo, hi = max(t0, tg.TS0), min(t1, tg.TS0 + tg.FIVE_YEARS)
    return share * max(0, hi - lo) / tg.FIVE_YEARS


def test_predicate_sizes_are_log_uniform():
    sp = tg.BaseSpec()
    preds = tg.make_predicates(sp, 4096, 1_000, 4_000_000, seed=1)
    assert len(preds) == 4096
    exp = np.array([expected_rows(sp, p) for p in preds])
    assert exp.min() > 0.9 * 1_000 and exp.max() < 1.1 * 4_000_000
    # log-uniform: each decade of [1e3, 4e6] holds its share of predicates
    logs = np.log(exp)
    frac_low = np.mean(exp < 1e4)
    assert abs(frac_low - np.log(10) / np.log(4000)) < 0.04
    assert abs(np.median(logs) - 0.5 * (np.log(1e3) + np.log(4e6))) < 0.15
    for tags, t0, t1 in preds:
        assert tags == sorted(set(tags)) and 1 <= len(tags) <= 8
        assert tg.TS0 <= t0 < t1 <= tg.TS0 + tg.FIVE_YEARS


def test_base_table_columns():
    sp = tg.BaseSpec(rows=400_000, nodes=50_000, tags=100)
    src, dst, ts, tag = (c.numpy() for c in tg.make_base_table(sp, seed=3))
    assert src.dtype == np.int32 and ts.dtype == np.int64 and tag.dtype == np.int32
    assert ts.min() >= tg.TS0 and ts.max() < tg.TS0 + tg.FIVE_YEARS
    assert tag.min() >= 0 and tag.max() < sp.tags
    # Zipf(1) tag shares: the top tag holds 1/H_100 of the rows
    share = np.bincount(tag, minlength=sp.tags) / sp.rows
    want = tg.tag_row_counts(sp) / sp.rows
    assert np.abs(share - want).max() < 0.01
    # ts uniform: each fifth of the window holds about a fifth of the rows
    q = np.bincount((ts - tg.TS0) * 5 // tg.FIVE_YEARS, minlength=5) / sp.rows
    assert np.abs(q - 0.2).max() < 0.01
    again = tg.make_base_table(sp, seed=3)
    assert np.array_equal(again[3].numpy(), tag) and np.array_equal(again[2].numpy(), ts)
