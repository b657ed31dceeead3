"""Seeded synthetic edge tables shaped like the paper's workloads.

This module is shared input plumbing: it feeds the same arrays to the CUDA
path and to the oracle, and it holds none of the conversion's arithmetic.

Every row is a pure function of (seed, row index), built only from integer
operations (hashes, masks, integer multiply with products below 2**63, and
``searchsorted`` over int64 thresholds), so a table generated on the CPU and
on the GPU is the same table bit for bit, and generation can be chunked.

Shapes (the paper's Table 2 gives the real graphs; these are stand-ins):

* ``tiny``    1M rows, 100K distinct non-negative 31-bit IDs, src Zipf(1.1)
              over a random ranking of the IDs, dst uniform, 5% exact
              duplicate rows, 0.1% self-loops.
* ``lj``      LiveJournal shape: 69M rows, 4.85M IDs, per-node out- and
              in-weights from a truncated power law (exponent 2.3, max
              20K, mean 69M/4.85M), rows drawn Chung-Lu style, 1% duplicates.
* ``twitter`` Twitter2010 shape: 1.47B rows, 41.7M IDs, Zipf rank weights
              with exponent 0.72 for in-edges (max in-degree about 3M) and
              0.5 for out-edges (max about 110K), 0.5% duplicates.

Rows are i.i.d. draws, so they are already in random order; a duplicate row
re-draws the row of another random index.
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np
import torch

M32 = 0xFFFFFFFF
M31 = 0x7FFFFFFF
TWO32 = 1 << 32

# odd multipliers below 2**31, so x * c stays below 2**63 for x < 2**32
_MUL = (0x7FEB352D, 0x6C8E9CF5, 0x5BD1E995 & M31 | 1, 0x27D4EB2F, 0x165667B1, 0x2545F491)


def _splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> tuple[int, int]:
    h = _splitmix64((seed << 16) ^ stream)
    return h & M32, (h >> 32) & M32


def _hash32(x: torch.Tensor) -> torch.Tensor:
    """32-bit integer mix on int64 tensors holding values in [0, 2**32)."""
    x = x ^ (x >> 16)
    x = (x * _MUL[0]) & M32
    x = x ^ (x >> 15)
    x = (x * _MUL[1]) & M32
    x = x ^ (x >> 16)
    return x


def uniform32(idx: torch.Tensor, seed: int, stream: int) -> torch.Tensor:
    """Counter-based uniform draw in [0, 2**32) for each index (int64)."""
    ka, kb = stream_key(seed, stream)
    return _hash32(_hash32((idx & M32) ^ ka) ^ kb ^ ((idx >> 32) & M32))


def perm_bits(x: torch.Tensor, bits: int, seed: int, stream: int) -> torch.Tensor:
    """A bijection on [0, 2**bits) (bits <= 31): rounds of odd multiply, key
    add and xor-shift, each invertible modulo 2**bits."""
    mask = (1 << bits) - 1
    for r in range(4):
        ka, kb = stream_key(seed, stream * 8 + r)
        x = (x * (_MUL[(r + 2) % len(_MUL)] | 1)) & mask
        x = (x + ka) & mask
        x = x ^ (x >> max(1, bits // 2))
        x = (x * ((kb & M31) | 1)) & mask
        x = x ^ (x >> max(1, (bits + 2) // 3))
    return x


def perm_range(x: torch.Tensor, n: int, seed: int, stream: int) -> torch.Tensor:
    """A bijection on [0, n) by cycle-walking a power-of-two bijection."""
    bits = max(1, int(n - 1).bit_length())
    y = perm_bits(x, bits, seed, stream)
    for _ in range(256):
        bad = y >= n
        if not bool(bad.any()):
            return y
        y = torch.where(bad, perm_bits(y, bits, seed, stream), y)
    raise RuntimeError("cycle walk did not settle")


def distinct_ids(n: int, seed: int, device) -> torch.Tensor:
    """n distinct non-negative 31-bit IDs (a keyed bijection of 0..n-1)."""
    i = torch.arange(n, dtype=torch.int64, device=device)
    return perm_bits(i, 31, seed, 901)


# ---------------------------------------------------------------- weights --
def thresholds_from_weights(w: np.ndarray) -> np.ndarray:
    """int64 cumulative thresholds in [0, 2**32]; a draw u in [0, 2**32)
    maps to slot searchsorted(T, u, right=True), with probability w/sum(w)
    up to 2**-32 rounding."""
    c = np.cumsum(w, dtype=np.float64)
    t = np.floor(c / c[-1] * TWO32).astype(np.int64)
    t[-1] = TWO32
    return t


@functools.lru_cache(maxsize=8)
def zipf_thresholds(n: int, s: float) -> np.ndarray:
    r = np.arange(1, n + 1, dtype=np.float64)
    return thresholds_from_weights(r ** (-s))


def _u01_np(n: int, seed: int, stream: int) -> np.ndarray:
    u = uniform32(torch.arange(n, dtype=torch.int64), seed, stream).numpy()
    return (u.astype(np.float64) + 0.5) / TWO32


def truncated_powerlaw(n: int, gamma: float, kmax: float, mean: float, seed: int,
                       stream: int) -> np.ndarray:
    """Per-node weights with P(k) ~ k**-gamma on [kmin, kmax]; kmin is found
    by bisection so that the weights average ``mean``."""
    a = gamma - 1.0
    u = _u01_np(n, seed, stream)

    def draw(kmin: float) -> np.ndarray:
        q = (kmin / kmax) ** a
        return kmin * (1.0 - u * (1.0 - q)) ** (-1.0 / a)

    lo, hi = 0.01, mean
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if draw(mid).mean() < mean:
            lo = mid
        else:
            hi = mid
    return draw(0.5 * (lo + hi))


@functools.lru_cache(maxsize=8)
def powerlaw_thresholds(n: int, gamma: float, kmax: float, mean: float, seed: int,
                        stream: int) -> np.ndarray:
    return thresholds_from_weights(truncated_powerlaw(n, gamma, kmax, mean, seed, stream))


# ----------------------------------------------------------------- tables --
@dataclasses.dataclass(frozen=True)
class TableSpec:
    name: str
    rows: int
    nodes: int
    out_law: tuple      # ("zipf", s) | ("powerlaw", gamma, kmax) | ("uniform",)
    in_law: tuple
    dup: float          # fraction of rows that repeat another row
    loop: float         # fraction of rows turned into self-loops

    def scaled(self, rows: int) -> "TableSpec":
        """Same shape with fewer rows; nodes shrink in proportion."""
        f = rows / self.rows
        nodes = max(16, int(round(self.nodes * f)))
        laws = []
        for law in (self.out_law, self.in_law):
            if law[0] == "powerlaw":
                law = ("powerlaw", law[1], max(8.0, law[2] * f ** 0.5))
            laws.append(law)
        return dataclasses.replace(self, name=f"{self.name}@{rows}", rows=rows, nodes=nodes,
                                   out_law=laws[0], in_law=laws[1])


SPECS = {
    "tiny": TableSpec("tiny", 1_000_000, 100_000, ("zipf", 1.1), ("uniform",), 0.05, 0.001),
    "lj": TableSpec("lj", 69_000_000, 4_850_000, ("powerlaw", 2.3, 20_000.0),
                    ("powerlaw", 2.3, 20_000.0), 0.01, 0.0),
    "twitter": TableSpec("twitter", 1_470_000_000, 41_700_000, ("zipf", 0.5), ("zipf", 0.72),
                         0.005, 0.0),
}


def _law_tables(spec: TableSpec, law: tuple, seed: int, stream: int, device):
    """(thresholds or None, slot -> node-number map or None)."""
    kind = law[0]
    if kind == "uniform":
        return None, None
    if kind == "zipf":
        t = torch.from_numpy(zipf_thresholds(spec.nodes, float(law[1]))).to(device)
        slot = torch.arange(spec.nodes, dtype=torch.int64, device=device)
        return t, perm_range(slot, spec.nodes, seed, stream)      # rank -> node
    if kind == "powerlaw":
        mean = spec.rows / spec.nodes
        t = torch.from_numpy(powerlaw_thresholds(spec.nodes, float(law[1]), float(law[2]),
                                                 mean, seed, stream)).to(device)
        return t, None                                            # slot = node
    raise ValueError(kind)


def _draw(u: torch.Tensor, nodes: int, tables) -> torch.Tensor:
    t, rank_map = tables
    if t is None:
        return (u * nodes) >> 32
    slot = torch.searchsorted(t, u, right=True)
    slot = torch.clamp(slot, max=nodes - 1)
    return slot if rank_map is None else rank_map[slot]


def make_table(spec: TableSpec | str, seed: int = 1, device="cpu", chunk: int = 1 << 25,
               start: int = 0, count: int | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """Generate (src, dst) int32 columns of ``spec`` on ``device``.

    ``start``/``count`` select rows [start, start+count) of the full table
    (every row is a function of its index, so a slice equals the same rows
    of the whole table)."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    device = torch.device(device)
    n = spec.rows
    if count is None:
        count = n - start
    if start < 0 or count < 0 or start + count > n:
        raise ValueError("row range outside the table")
    ids = distinct_ids(spec.nodes, seed, device)
    out_tab = _law_tables(spec, spec.out_law, seed, 11, device)
    in_tab = _law_tables(spec, spec.in_law, seed, 12, device)
    src = torch.empty(count, dtype=torch.int32, device=device)
    dst = torch.empty(count, dtype=torch.int32, device=device)
    dup_cut = int(spec.dup * TWO32)
    loop_cut = int(spec.loop * TWO32)
    for lo in range(start, start + count, chunk):
        hi = min(start + count, lo + chunk)
        i = torch.arange(lo, hi, dtype=torch.int64, device=device)
        # a duplicate row copies the base draw of another random row index
        is_dup = uniform32(i, seed, 1) < dup_cut
        j = torch.where(is_dup, (uniform32(i, seed, 2) * n) >> 32, i)
        s = ids[_draw(uniform32(j, seed, 3), spec.nodes, out_tab)]
        d = ids[_draw(uniform32(j, seed, 4), spec.nodes, in_tab)]
        if loop_cut:
            d = torch.where(uniform32(j, seed, 5) < loop_cut, s, d)
        src[lo - start:hi - start] = s.to(torch.int32)
        dst[lo - start:hi - start] = d.to(torch.int32)
    return src, dst


def signed_table(rows: int, nodes: int, seed: int = 1, device="cpu") -> tuple:
    """Rows over IDs spread across the whole signed int32 range (negative
    IDs, INT32_MIN and INT32_MAX included), Zipf(1.0) sources, uniform
    destinations, some duplicates and self-loops."""
    device = torch.device(device)
    i = torch.arange(nodes, dtype=torch.int64, device=device)
    ids = (perm_bits(i, 31, seed, 77) * 2 + (uniform32(i, seed, 78) & 1)) - (1 << 31)
    ids[0] = -(1 << 31)
    if nodes > 1:
        ids[1] = (1 << 31) - 1
    spec = TableSpec("signed", rows, nodes, ("zipf", 1.0), ("uniform",), 0.03, 0.01)
    out_tab = _law_tables(spec, spec.out_law, seed, 21, device)
    r = torch.arange(rows, dtype=torch.int64, device=device)
    is_dup = uniform32(r, seed, 22) < int(0.03 * TWO32)
    j = torch.where(is_dup, (uniform32(r, seed, 23) * rows) >> 32, r)
    s = ids[_draw(uniform32(j, seed, 24), nodes, out_tab)]
    d = ids[_draw(uniform32(j, seed, 25), nodes, (None, None))]
    d = torch.where(uniform32(j, seed, 26) < int(0.01 * TWO32), s, d)
    return s.to(torch.int32), d.to(torch.int32)


# ------------------------------------------------------------ base tables --
FIVE_YEARS = 5 * 365 * 24 * 3600
TS0 = 1_420_070_400  # 2015-01-01T00:00:00Z, seconds


@dataclasses.dataclass(frozen=True)
class BaseSpec:
    """A resident base table {src, dst, ts, tag}: src/dst drawn Chung-Lu style
    from truncated power-law weights (as in the LiveJournal shape), ts uniform
    over five years (seconds), tag Zipf(s) over `tags` values."""
    rows: int = 200_000_000
    nodes: int = 16_000_000
    tags: int = 10_000
    tag_s: float = 1.0


def make_base_table(spec: BaseSpec = BaseSpec(), seed: int = 1, device="cpu",
                    chunk: int = 1 << 25):
    device = torch.device(device)
    edge = TableSpec("base", spec.rows, spec.nodes, ("powerlaw", 2.3, 20_000.0),
                     ("powerlaw", 2.3, 20_000.0), 0.0, 0.0)
    src, dst = make_table(edge, seed=seed, device=device, chunk=chunk)
    ts = torch.empty(spec.rows, dtype=torch.int64, device=device)
    tag = torch.empty(spec.rows, dtype=torch.int32, device=device)
    tag_t = torch.from_numpy(zipf_thresholds(spec.tags, spec.tag_s)).to(device)
    for lo in range(0, spec.rows, chunk):
        hi = min(spec.rows, lo + chunk)
        i = torch.arange(lo, hi, dtype=torch.int64, device=device)
        ts[lo:hi] = TS0 + ((uniform32(i, seed, 41) * FIVE_YEARS) >> 32)
        tag[lo:hi] = torch.clamp(torch.searchsorted(tag_t, uniform32(i, seed, 42), right=True),
                                 max=spec.tags - 1).to(torch.int32)
    return src, dst, ts, tag


def tag_row_counts(spec: BaseSpec) -> np.ndarray:
    """Expected rows per tag (Zipf shares of the row count)."""
    r = np.arange(1, spec.tags + 1, dtype=np.float64)
    w = r ** (-spec.tag_s)
    return spec.rows * w / w.sum()


def make_predicates(spec: BaseSpec, npred: int, lo: int, hi: int, seed: int = 1,
                    max_tags: int = 8):
    """Predicates (tags, t0, t1) whose expected selection sizes are
    log-uniform in [lo, hi]: tags are added in a random order until their rows
    reach the target, then the time window is the matching fraction of five
    years at a random start."""
    rng = np.random.default_rng(seed)
    counts = tag_row_counts(spec)
    preds = []
    for _ in range(npred):
        target = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        order = rng.integers(0, spec.tags, 4 * max_tags)
        tags, total = [], 0.0
        for t in order:
            if total >= target or len(tags) >= max_tags:
                break
            if int(t) in tags:
                continue
            tags.append(int(t))
            total += counts[t]
        if total < target:  # take the biggest tags instead
            tags = [int(t) for t in np.argsort(-counts)[:max_tags]]
            total = float(counts[tags].sum())
        frac = min(1.0, target / total)
        span = max(1, int(frac * FIVE_YEARS))
        t0 = TS0 + int(rng.integers(0, max(1, FIVE_YEARS - span + 1)))
        preds.append((sorted(tags), t0, t0 + span))
    return preds
