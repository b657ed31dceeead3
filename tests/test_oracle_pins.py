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
