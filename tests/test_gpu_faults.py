"""Failure detection without a GPU fault.

The failures are made on the host through the library's test hooks, and
nothing on the device faults, traps or waits without bound:
  * a bounded device wait that runs out: the next conversion's first radix
    pass never claims its tile 0, so the tiles after it wait on it until a
    lowered spin bound (a few thousand polls) and record an error; the call
    returns RINGO_ETIMEOUT, frees what it holds, and the device keeps working;
  * device allocations that fail one after another at every point of a
    conversion, a batch and a served request: each returns RINGO_ENOMEM and
    the library's pool is back at its baseline afterwards (nothing leaks).
"""
import time

import numpy as np
import pytest
import torch

import oracle
import pins
from paper_1503_07881_gb300 import ringo, tablegen as tg

pytestmark = pytest.mark.gpu


def _pool_used() -> int:
    torch.cuda.synchronize()
    return ringo.ringo_test_pool_used()


def _oracle(src, dst):
    return oracle.table_to_graph(src.cpu().numpy(), dst.cpu().numpy())


def test_lookback_wait_runs_out_and_device_keeps_working():
    src, dst = tg.make_table(tg.SPECS["lj"].scaled(300_000), seed=41, device="cuda")
    want = _oracle(src, dst)
    ringo.ringo_table_to_graph(src, dst).free()  # warm: pool and kernels loaded
    base = _pool_used()
    for spin_limit in (1024, 4096):
        ringo.ringo_test_inject_lookback_timeout(spin_limit)
        t0 = time.monotonic()
        with pytest.raises(ringo.RingoError) as ei:
            ringo.ringo_table_to_graph(src, dst)
        assert ei.value.status == ringo.RINGO_ETIMEOUT
        assert "bounded device wait" in str(ei.value)
        assert time.monotonic() - t0 < 30.0
        assert _pool_used() == base
        # the device still answers and the next conversion is exact
        g = ringo.ringo_table_to_graph(src, dst)
        got = g.copy_to_host()
        g.free()
        pins.assert_same_graph(got, want, f"after a timeout at {spin_limit} spins")
    assert _pool_used() == base


def test_conversion_allocation_failures_return_enomem_without_leaks():
    src, dst = tg.make_table(tg.SPECS["tiny"].scaled(200_000), seed=42, device="cuda")
    want = _oracle(src, dst)
    ringo.ringo_table_to_graph(src, dst).free()
    base = _pool_used()
    failed = 0
    try:
        for skip in range(12):
            ringo.ringo_test_inject_alloc_failure(skip)
            try:
                g = ringo.ringo_table_to_graph(src, dst)
            except ringo.RingoError as e:
                assert e.status == ringo.RINGO_ENOMEM, str(e)
                assert "injected" in str(e)
                failed += 1
            else:
                ringo.ringo_test_inject_alloc_failure(-1)
                got = g.copy_to_host()
                g.free()
                pins.assert_same_graph(got, want, f"after {skip} allocations")
            assert _pool_used() == base, f"pool not back at its baseline after {skip} allocations"
    finally:
        ringo.ringo_test_inject_alloc_failure(-1)
    # the workspace, both neighbour arrays, the node arrays and the rank maps
    assert failed >= 7


def _small_base(seed=43):
    spec = tg.BaseSpec(rows=300_000, nodes=40_000, tags=200)
    cols = tg.make_base_table(spec, seed=seed)
    preds = tg.make_predicates(spec, 24, 100, 30_000, seed=seed)
    src, dst, ts, tag = (c.cuda() for c in cols)
    return ringo.BaseTable(src, dst, ts, tag), [c.numpy() for c in cols], preds


def test_batch_allocation_failures_return_enomem_without_leaks():
    base_t, cols, preds = _small_base()
    try:
        ref = base_t.convert_batch(preds)
        want = [ref.copy_to_host(i) for i in range(len(preds))]
        ref.free()
        base = _pool_used()
        failed = 0
        for skip in range(8):
            ringo.ringo_test_inject_alloc_failure(skip)
            try:
                bt = base_t.convert_batch(preds)
            except ringo.RingoError as e:
                assert e.status == ringo.RINGO_ENOMEM, str(e)
                failed += 1
            else:
                ringo.ringo_test_inject_alloc_failure(-1)
                for i in range(len(preds)):
                    pins.assert_same_graph(bt.copy_to_host(i), want[i], f"graph {i}")
                bt.free()
            assert _pool_used() == base, f"pool not back at its baseline after {skip} allocations"
        assert failed >= 1
    finally:
        ringo.ringo_test_inject_alloc_failure(-1)
        base_t.free()


def test_served_request_allocation_failure_is_reported_and_serving_goes_on():
    base_t, cols, preds = _small_base(seed=44)
    server = ringo.Server(base_t, 2 << 30)
    try:
        alone = server.wait(server.submit(preds[0], topk=10))
        assert alone["status"] == ringo.RINGO_OK
        base = _pool_used()
        for skip in range(3):
            ringo.ringo_test_inject_alloc_failure(skip)
            r = server.wait(server.submit(preds[0], topk=10))
            ringo.ringo_test_inject_alloc_failure(-1)
            assert r["status"] in (ringo.RINGO_OK, ringo.RINGO_ENOMEM)
            if r["status"] == ringo.RINGO_OK:
                for d in ("topk_out", "topk_in"):
                    assert np.array_equal(r[d][0], alone[d][0])
            assert _pool_used() == base
        r0 = server.wait(server.submit(preds[0], topk=10))
        ringo.ringo_test_inject_alloc_failure(0)
        failed = server.wait(server.submit(preds[1], topk=10))
        ringo.ringo_test_inject_alloc_failure(-1)
        assert failed["status"] == ringo.RINGO_ENOMEM
        again = server.wait(server.submit(preds[0], topk=10))
        assert again["status"] == ringo.RINGO_OK
        for d in ("topk_out", "topk_in"):
            assert np.array_equal(again[d][0], r0[d][0]) and np.array_equal(again[d][1], r0[d][1])
        assert _pool_used() == base
    finally:
        ringo.ringo_test_inject_alloc_failure(-1)
        server.close()
        base_t.free()
