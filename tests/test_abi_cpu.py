"""The C-ABI library builds, loads and exports every declared symbol, and
argument checks that happen before any CUDA call behave (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1503_07881_gb300 import build, ringo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols() -> set:
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"RINGO_API\s+[\w\s\*]*?\b(ringo_\w+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 17
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() == set(ringo.SIGNATURES)


def test_status_strings_and_version():
    lib = ringo.load()
    assert lib.ringo_status_string(0) == b"ok"
    assert lib.ringo_status_string(4) == b"device wait timed out"
    assert lib.ringo_version().startswith(b"ringo-gb300")


def test_argument_validation_before_any_device_work():
    lib = ringo.load()
    h = ctypes.c_void_p()
    assert lib.ringo_table_to_graph(None, None, 0, None, None) == ringo.RINGO_EINVAL
    assert lib.ringo_table_to_graph(None, None, -1, None, ctypes.byref(h)) == ringo.RINGO_EINVAL
    assert lib.ringo_table_to_graph(None, None, 5, None, ctypes.byref(h)) == ringo.RINGO_EINVAL
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.ringo_table_to_graph(fake, fake, 1 << 31, None, ctypes.byref(h)) == ringo.RINGO_ERANGE
    assert h.value is None
    assert b"nrows" in lib.ringo_last_error()
    v = ctypes.c_int64()
    assert lib.ringo_graph_num_nodes(None, ctypes.byref(v)) == ringo.RINGO_EINVAL
    lib.ringo_graph_free(None)  # no-op


def test_undirected_row_limit_checked_before_any_device_work():
    lib = ringo.load()
    fake = ctypes.c_void_p(4096)  # never dereferenced: the size check comes first
    h = ctypes.c_void_p()
    rc = lib.ringo_table_to_undirected_graph(fake, fake, 1 << 31, None, ctypes.byref(h))
    assert rc == ringo.RINGO_ERANGE and not h.value
    assert b"nrows" in lib.ringo_last_error()


def test_failure_injection_hooks_argument_handling():
    """The test hooks check their arguments before arming anything (the
    failures they make are exercised on the GPU in test_gpu_faults.py)."""
    lib = ringo.load()
    assert lib.ringo_test_inject_lookback_timeout(0) == ringo.RINGO_EINVAL
    assert lib.ringo_test_inject_lookback_timeout((1 << 21) + 1) == ringo.RINGO_EINVAL
    assert b"spin_limit" in lib.ringo_last_error()
    assert lib.ringo_test_pool_used(None) == ringo.RINGO_EINVAL
    # arming and disarming the allocation failure touches no device
    assert lib.ringo_test_inject_alloc_failure(3) == ringo.RINGO_OK
    assert lib.ringo_test_inject_alloc_failure(-1) == ringo.RINGO_OK


def test_sort_opts_force_argument_checks():
    """Forcing pass options checks their ranges before anything else; a
    valid force and its release touch no device."""
    lib = ringo.load()
    for bad in ((3, 1, 0), (-1, 1, 0), (0, 3, 0), (0, -1, 0), (0, 1, -5), (0, 1, 0, 7),
                (0, 1, 0, 10), (0, 1, 0, -1)):
        o = ringo.SortOpts(*bad)
        assert lib.ringo_sort_opts_force(ctypes.byref(o)) == ringo.RINGO_EINVAL, bad
    for good in ((2, 2, 0, 9), (1, 0, 0, 8), (0, 1, 0, 0)):
        o = ringo.SortOpts(*good)
        assert lib.ringo_sort_opts_force(ctypes.byref(o)) == ringo.RINGO_OK, good
    o = ringo.SortOpts(1, 2, 0)
    assert lib.ringo_sort_opts_force(ctypes.byref(o)) == ringo.RINGO_OK
    assert lib.ringo_sort_opts_force(None) == ringo.RINGO_OK
    assert lib.ringo_tune_lookup(3, 10, ctypes.byref(o), None) == ringo.RINGO_EINVAL
    assert lib.ringo_tune_table(None, None, 10, None, ctypes.byref(o), None) == ringo.RINGO_EINVAL


def test_tune_cache_rejects_a_file_that_is_not_a_cache(tmp_path):
    lib = ringo.load()
    bad = tmp_path / "not_a_cache.json"
    bad.write_text('{"something": 1}')
    assert lib.ringo_tune_set_cache(str(bad).encode()) == ringo.RINGO_EINVAL
    assert lib.ringo_tune_set_cache(None) == ringo.RINGO_OK


def test_tune_cache_keeps_pass_options_and_repairs_bad_ones(tmp_path):
    """A cache file's entries survive being read and written back: the rank
    method, prefetch distance and in-direction digit width of each; values
    out of range come back as the defaults.  No device is touched."""
    import json
    lib = ringo.load()
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"version": 1, "entries": [
        {"gpu": 'GPU "A"', "kind": 0, "size_class": 30, "rank_method": 2, "prefetch_waves": 0,
         "in_digit_bits": 9, "wave_rows": 0, "ms": 1.5, "out_passes": 8, "in_passes": 3},
        {"gpu": "GPU B", "kind": 1, "size_class": 20, "rank_method": 7, "prefetch_waves": 5,
         "in_digit_bits": 11, "wave_rows": 4096, "ms": 2.0, "out_passes": 8, "in_passes": 4}]}))
    try:
        assert lib.ringo_tune_set_cache(str(path).encode()) == ringo.RINGO_OK
        entries = {(e["gpu"], e["kind"], e["size_class"]): e
                   for e in json.loads(path.read_text())["entries"]}
        a = entries[('GPU "A"', 0, 30)]
        assert (a["rank_method"], a["prefetch_waves"], a["in_digit_bits"]) == (2, 0, 9)
        assert a["in_passes"] == 3
        b = entries[("GPU B", 1, 20)]
        assert (b["rank_method"], b["prefetch_waves"], b["in_digit_bits"]) == (0, 1, 8)
        assert b["wave_rows"] == 4096
    finally:
        assert lib.ringo_tune_set_cache(None) == ringo.RINGO_OK
