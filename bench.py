"""Benchmark: table->graph conversion throughput on GB300.

One step = one full conversion (every kernel of the path) of a synthetic edge
table already resident in HBM, through the C ABI (ringo_table_to_graph).
Default workload: the Twitter2010-shaped table (1.47B rows, 41.7M IDs), the
configuration the paper's headline conversion number is quoted on (its
Table 5).  edges/s = input rows / wall time, the paper's definition.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload twitter|lj|tiny]
    python bench.py --impl reference ...   # the CPU oracle on bounded samples

For N > 1 (torchrun) every rank converts its own table (replicas, weak
scaling); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

WORKLOADS = {
    "twitter": "Twitter2010-shaped edge table: 1.47B rows, 41.7M distinct 31-bit IDs, "
               "Zipf in-degree (s=0.72) and out-degree (s=0.5), 0.5% duplicates, random order",
    "lj": "LiveJournal-shaped edge table: 69M rows, 4.85M distinct 31-bit IDs, power-law "
          "out/in weights (exponent 2.3, max 20K), 1% duplicates, random order",
    "tiny": "1M-row edge table, 100K distinct 31-bit IDs, Zipf(1.1) src, uniform dst, "
            "5% duplicates, 0.1% self-loops",
    "batched": "resident 200M-row base table {src, dst int32 Chung-Lu over 16M IDs, ts int64 "
               "uniform over 5 years, tag int32 Zipf over 10K}; 4096 tag/time-window "
               "selections, sizes log-uniform 1K-4M rows, converted as one batch",
    "served": "the same resident base table; open-loop Poisson select+convert+top-k(100) "
              "requests, sizes log-uniform 10K-50M rows, 120 GB budget",
}
# the paper's own table->graph rates (Table 5, 4x Xeon E7-4870, real graphs)
PAPER_RATE = {"twitter": 18.0e6, "lj": 13.0e6}
CPU_SAMPLE_ROWS = {"twitter": 2_000_000, "lj": 2_000_000, "tiny": 1_000_000}
REF_SAMPLE_ROWS = {"twitter": 1_000_000, "lj": 1_000_000, "tiny": 250_000}
SORT_SOURCES = ["paper_1503_07881_gb300/csrc/sort_kernels.cu",
                "paper_1503_07881_gb300/csrc/ringo_internal.cuh",
                "paper_1503_07881_gb300/csrc/device_util.cuh"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ dist --
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- roofline ---
def host_cpu() -> dict:
    """The host the CPU baseline ran on: logical cores and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def measured_peak_hbm() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def sort_source_digest() -> str:
    h = hashlib.sha256()
    for p in SORT_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_key_pass() -> float | None:
    """DRAM bytes per key per radix pass from the committed ncu figures
    (profiles/sweep_traffic.json, written beside the ncu summary), if they
    were taken on the current sort source."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        per_key = float(rec["dram_bytes_per_key_pass"])
        digest = str(rec["source_digest"])
    except (OSError, KeyError, ValueError, TypeError):
        return None
    return per_key if digest == sort_source_digest() else None


# --------------------------------------------------------------- our arm --
def run_ours(args, world, rank, local):
    from paper_1503_07881_gb300 import ringo, tablegen
    import oracle

    ringo.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = tablegen.SPECS[args.workload]
    t0 = time.time()
    src, dst = tablegen.make_table(spec, seed=args.seed + rank, device=dev)
    torch.cuda.synchronize()
    log(f"[rank {rank}] generated {spec.rows} rows in {time.time() - t0:.1f}s")
    N = spec.rows

    def step():
        g = ringo.ringo_table_to_graph(src, dst)
        info = g.info()
        g.free()
        return info

    info = None
    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    E, V = info["num_edges"], info["num_nodes"]
    P_out, P_in = info["out_sort_passes"], info["in_sort_passes"]

    sampler = ClockSampler(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    sampler.start()
    ringo.ringo_profile_start()
    start.record(stream)
    for _ in range(args.steps):
        step()
    end.record(stream)
    torch.cuda.synchronize()
    prof = ringo.ringo_profile_stop()
    clocks = sampler.stop()
    barrier(world)
    ms = start.elapsed_time(end) / args.steps
    ms = max_over_ranks(ms, world)
    value = N * world / (ms / 1e3)

    # roofline of the dominant kernel (the onesweep radix pass)
    peak, peak_kind = measured_peak_hbm()
    by = {p["name"]: p for p in prof}
    sw = by.get("onesweep")
    moved = 16.0 * (N * P_out + E * P_in) * args.steps  # read + write of 8-byte keys
    sw_ms = sw["total_ms"] if sw else float("nan")
    achieved = moved / (sw_ms / 1e3) / 1e9
    per_key = ncu_traffic_per_key_pass()
    traffic = None if per_key is None else per_key * N  # one out-sort launch over N keys
    kernel_share = {p["name"]: round(p["total_ms"] / (ms * args.steps), 4) for p in prof}
    # whole-path frozen model (8N + 20V + 16 + 8E compulsory, + 104N + 64E sort model)
    model_bytes = 8 * N + 20 * V + 16 + 8 * E + 104 * N + 64 * E
    model_frac = model_bytes / (ms / 1e3) / 1e9 / peak

    # e2e: host columns -> graph -> host arrays, through the C ABI
    e2e = None
    if not args.no_e2e:
        torch.cuda.empty_cache()
        hs = torch.empty(N, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(N, dtype=torch.int32, pin_memory=True)
        hs.copy_(src)
        hd.copy_(dst)
        outs = {"node_ids": torch.empty(V, dtype=torch.int32, pin_memory=True),
                "out_off": torch.empty(V + 1, dtype=torch.int64, pin_memory=True),
                "out_nbr": torch.empty(E, dtype=torch.int32, pin_memory=True),
                "in_off": torch.empty(V + 1, dtype=torch.int64, pin_memory=True),
                "in_nbr": torch.empty(E, dtype=torch.int32, pin_memory=True)}

        split = {"host_io_call_ms": 0.0}

        def e2e_step(record=False):
            # host columns -> host arrays in one call; the out-CSR comes back
            # while the in-CSR is built
            t0 = time.perf_counter()
            got = ringo.ringo_table_to_graph_host_io(hs, hd, out=outs)
            assert got["num_edges"] == E and got["num_nodes"] == V
            if record:
                split["host_io_call_ms"] += (time.perf_counter() - t0) * 1e3

        e2e_step()
        torch.cuda.synchronize()
        k2 = max(1, min(args.steps, 5))
        barrier(world)
        s2 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        ringo.ringo_profile_start()
        s2.record(stream)
        for _ in range(k2):
            e2e_step(record=True)
        e2.record(stream)
        torch.cuda.synchronize()
        for p in ringo.ringo_profile_stop():  # copy steps of the call, per step
            if p["name"] in ("host:input_alloc", "input_h2d", "out_csr_d2h", "in_csr_d2h"):
                split[p["name"] + "_ms"] = p["total_ms"]
        ms2 = max_over_ranks(s2.elapsed_time(e2) / k2, world)
        e2e = {"value": N * world / (ms2 / 1e3), "unit": "edges/s", "ms_per_step": round(ms2, 3),
               "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 4 * V + 16 * (V + 1) + 8 * E,
               "api": "ringo_table_to_graph_host_io (pinned host columns in, pinned host "
                      "arrays out; out-CSR copied back during the in-sort)",
               "host_split_ms": {k: round(v / k2, 2) for k, v in split.items()}}
        del hs, hd, outs

    # graph -> table (Section 3.4) and PageRank (Table "paralg") on the same graph
    to_table = pagerank = triangles = table_ops = None
    if not args.no_to_table:
        table_ops = run_select_join(args, src, dst, stream)
        to_table, pagerank = run_graph_ops(args, src, dst, stream, peak, peak_kind)
        if world == 1:
            triangles = run_triangles(args, stream, src, dst)

    # CPU baseline: the oracle on a bounded prefix sample of the same table
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        S = min(N, CPU_SAMPLE_ROWS[args.workload])
        s_h, d_h = src[:S].cpu().numpy(), dst[:S].cpu().numpy()
        t1 = time.perf_counter()
        oracle.table_to_graph(s_h, d_h)
        dt = time.perf_counter() - t1
        cpu = {"value": S / dt, "unit": "edges/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"first {S} rows of the same table, one oracle run "
                         f"(std::sort + std::unique + std::map), {dt:.1f}s"}

    launches = sum(p["launches"] for p in prof)
    batched = served = None
    if world == 1 and not (args.no_batched and args.no_served):
        del src, dst
        torch.cuda.empty_cache()
        batched, served = run_base_workloads(args)
    line = {
        "metric": "table->graph edges/s",
        "value": value,
        "unit": "edges/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (value / PAPER_RATE[args.workload]) if args.workload in PAPER_RATE else None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "rows": N, "distinct_edges": E,
                   "nodes": V, "radix_passes": {"out": P_out, "in": P_in},
                   "l2": "inputs (8 B/row) larger than L2", "seed": args.seed,
                   "parallelism": f"replicas x{world}",
                   "model_roofline_frac": round(model_frac, 4),
                   "model_bytes_per_step": model_bytes,
                   "kernel_time_share": kernel_share,
                   "vs_baseline_note": "paper Table 5 rate on real graphs, 4x Xeon E7-4870"},
        "roofline": {"bound": "hbm", "kernel": "onesweep radix pass",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind,
                     "algorithmic_bytes": "16 B per key per pass (8 B read + 8 B write)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "batched": batched,
        "served": served,
        "graph_to_table": to_table,
        "pagerank": pagerank,
        "triangles": triangles,
        "select_join": table_ops,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_base_only(args):
    """--workload batched|served: one JSON line for that form alone."""
    from paper_1503_07881_gb300 import ringo
    ringo.load()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    batched, served = run_base_workloads(args)
    clocks = sampler.stop()
    if args.workload == "batched":
        b = batched
        ok = b and "error" not in b
        line = {"metric": "table->graph edges/s, batched", "value": b["value"] if ok else None,
                "unit": "edges/s", "n_gpus": 1, "steps": args.batch_steps, "warmup": 1,
                "ms_per_step": b["ms_per_step"] if ok else None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOADS["batched"]}, "batched": b, "clocks": clocks}
    else:
        line = {"metric": "served select+convert+top-k latency and edges/s", "value": None,
                "unit": "edges/s", "n_gpus": 1, "higher_is_better": True, "dtype": "int32",
                "data": "synthetic", "config": {"workload": WORKLOADS["served"]},
                "served": served, "clocks": clocks}
        if served and "error" not in served:
            line["value"] = served["rates"][-1]["server"]["edges_per_s"]
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- graph -> table --
PAPER_TO_TABLE_RATE = {"twitter": 50.4e6, "lj": 46.0e6}  # Table 5, edges/s


PAPER_PAGERANK_S = {"twitter": 60.5, "lj": 2.76}  # Table "paralg", ten iterations


def run_graph_ops(args, src, dst, stream, peak, peak_kind) -> tuple[dict, dict]:
    """Graph -> table and PageRank on the graph of the workload."""
    from paper_1503_07881_gb300 import ringo
    g = ringo.ringo_table_to_graph(src, dst)
    try:
        return run_to_table(args, g, stream, peak, peak_kind), run_pagerank(args, g, stream, peak,
                                                                            peak_kind)
    finally:
        g.free()
        torch.cuda.empty_cache()


def run_pagerank(args, g, stream, peak, peak_kind) -> dict:
    """Ten PageRank iterations (d = 0.85), timed with CUDA events over 3 runs
    after one warm-up."""
    from paper_1503_07881_gb300 import ringo
    V, E = g.num_nodes, g.num_edges
    out = torch.empty(max(V, 1), dtype=torch.float64, device="cuda")
    iters, runs = 10, 3
    g.pagerank(0.85, iters, out=out)
    torch.cuda.synchronize()
    ringo.ringo_profile_start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(runs):
        g.pagerank(0.85, iters, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    prof = {p["name"]: p for p in ringo.ringo_profile_stop()}
    ms = a.elapsed_time(b) / runs
    total = float(out[:V].sum().item())
    # edge pass per iteration: in-neighbour index (4 B) and its contribution
    # (8 B) per edge, the in-offsets, one add per node
    edge_ms = prof["pagerank_edges"]["total_ms"] / (runs * iters) if "pagerank_edges" in prof else None
    algo = 12 * E + 8 * (V + 1) + 8 * V
    paper = PAPER_PAGERANK_S.get(args.workload)
    res = {"metric": "PageRank, 10 iterations", "ms": round(ms, 3), "unit": "ms",
           "iterations": iters, "damping": 0.85, "edges": E, "nodes": V,
           "edges_per_s": E * iters / (ms / 1e3), "rank_sum": total,
           "paper_s": paper, "vs_paper": (paper * 1e3 / ms) if paper else None,
           "dtype": "f64"}
    if edge_ms:
        res["roofline"] = {"bound": "hbm", "kernel": "k_pr_edges",
                           "achieved": algo / (edge_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": algo / (edge_ms / 1e3) / 1e9 / peak,
                           "algorithmic_bytes": "12 B per edge + 16 B per node",
                           "peak_source": peak_kind}
    del out
    return res


PAPER_TRIANGLES_S = {"lj": 6.13, "twitter": 263.6}  # Table "paralg"


def _triangles_of(src, dst, stream, runs: int) -> dict:
    from paper_1503_07881_gb300 import ringo
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    g = ringo.ringo_table_to_undirected_graph(src, dst)  # warm-up
    tri = g.count_triangles()
    g.free()
    torch.cuda.synchronize()
    ringo.ringo_profile_start()
    a.record(stream)
    g = ringo.ringo_table_to_undirected_graph(src, dst)
    b.record(stream)
    for _ in range(runs):
        t = g.count_triangles()
        assert t == tri
    c.record(stream)
    torch.cuda.synchronize()
    prof = {p["name"]: p["total_ms"] for p in ringo.ringo_profile_stop()}
    conv_ms = a.elapsed_time(b)
    count_ms = b.elapsed_time(c) / runs
    V, E = g.num_nodes, g.num_edges
    g.free()
    torch.cuda.empty_cache()
    merge_ms = prof.get("undirected_count", 0.0) + prof.get("undirected_write", 0.0)
    return {"triangles": tri, "nodes": V, "adjacency_entries": E,
            "undirected_conversion_ms": round(conv_ms, 3),
            "of_which_list_merge_ms": round(merge_ms, 3), "count_ms": round(count_ms, 3),
            "count_runs": runs}


def run_triangles(args, stream, src=None, dst=None) -> dict:
    """Undirected conversion (the directed conversion, then each node's out-
    and in-list merged) and triangle count of the LiveJournal-shaped table,
    and of the Twitter-shaped one when that is the workload (its resident
    table is reused)."""
    from paper_1503_07881_gb300 import tablegen
    out = {"metric": "undirected conversion and triangle count"}
    ls, ld = tablegen.make_table("lj", seed=args.seed, device="cuda")
    torch.cuda.synchronize()
    r = _triangles_of(ls, ld, stream, runs=3)
    del ls, ld
    r.update({"workload": WORKLOADS["lj"], "paper_s": PAPER_TRIANGLES_S["lj"],
              "vs_paper": PAPER_TRIANGLES_S["lj"] * 1e3 / r["count_ms"]})
    out["lj"] = r
    if args.workload == "twitter" and src is not None:
        r = _triangles_of(src, dst, stream, runs=1)
        r.update({"workload": WORKLOADS["twitter"], "paper_s": PAPER_TRIANGLES_S["twitter"],
                  "vs_paper": PAPER_TRIANGLES_S["twitter"] * 1e3 / r["count_ms"]})
        out["twitter"] = r
    return out


PAPER_TABLE_OPS_S = {"twitter": {"select_10k": 1.6, "select_all_but_10k": 1.6, "join_10k": 4.2,
                                   "join_all_but_10k": 29.7},
                     "lj": {"select_10k": 0.2, "select_all_but_10k": 0.1, "join_10k": 0.6,
                            "join_all_but_10k": 3.1}}  # Table "table_ringo"


def run_select_join(args, src, dst, stream) -> dict:
    """Section 4's table benchmark on the workload's edge table: select by
    comparison with a constant keeping 10K rows or all but 10K (in place), and
    join on src with a single-column table chosen so the output is about 10K
    rows or all but about 10K."""
    from paper_1503_07881_gb300 import ringo
    N = src.numel()
    k = 10_000
    srt = torch.sort(src).values
    lo_val = int(srt[k].item())  # src < lo_val keeps the k smallest rows (ties aside),
    #                              src >= lo_val all the others
    del srt
    # join keys: source IDs of a random node subset whose rows total about k
    ids, counts = torch.unique(src, return_counts=True)
    perm = torch.randperm(ids.numel(), device=ids.device, generator=torch.Generator(device=ids.device).manual_seed(5))
    csum = torch.cumsum(counts[perm], 0)
    take = int(torch.searchsorted(csum, torch.tensor(k, device=csum.device)).item()) + 1
    keys_small = ids[perm[:take]].contiguous()
    keys_large = ids[perm[take:]].contiguous()
    del ids, counts, perm, csum
    ws, wd = torch.empty_like(src), torch.empty_like(dst)
    out = {}

    splits = {}

    def timed(fn, runs=3, name=None):
        ms = []
        for r in range(runs + 1):
            ws.copy_(src)
            wd.copy_(dst)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if r:
                ringo.ringo_profile_start()
            a.record(stream)
            res = fn()
            b.record(stream)
            torch.cuda.synchronize()
            if r:
                ms.append(a.elapsed_time(b))
                for p in ringo.ringo_profile_stop():  # per-kernel device time, summed over runs
                    splits.setdefault(name, {}).setdefault(p["name"], 0.0)
                    splits[name][p["name"]] += p["total_ms"] / runs
        return res, statistics.median(ms)

    paper = PAPER_TABLE_OPS_S.get(args.workload, {})
    n1, ms1 = timed(lambda: ringo.ringo_table_select(ws, wd, 0, "<", lo_val), name="select_10k")
    n2, ms2 = timed(lambda: ringo.ringo_table_select(ws, wd, 0, ">=", lo_val), name="select_all_but_10k")
    cap = N
    js, jd = torch.empty_like(src), torch.empty_like(dst)

    def join(keys):
        import ctypes
        n = ctypes.c_int64()
        rc = ringo.load().ringo_table_join(src.data_ptr(), dst.data_ptr(), N, 0, keys.data_ptr(),
                                           keys.numel(), js.data_ptr(), jd.data_ptr(), cap,
                                           ctypes.byref(n), torch.cuda.current_stream().cuda_stream)
        assert rc == 0, rc
        return n.value

    n3, ms3 = timed(lambda: join(keys_small), name="join_10k")
    n4, ms4 = timed(lambda: join(keys_large), name="join_all_but_10k")
    for name, rows, ms, in_rows in (("select_10k", n1, ms1, N), ("select_all_but_10k", n2, ms2, N),
                                    ("join_10k", n3, ms3, N + keys_small.numel()),
                                    ("join_all_but_10k", n4, ms4, N + keys_large.numel())):
        p = paper.get(name)
        out[name] = {"ms": round(ms, 3), "output_rows": rows, "rows_per_s": in_rows / (ms / 1e3),
                     "input_rows": in_rows, "paper_s": p, "vs_paper": (p * 1e3 / ms) if p else None,
                     "kernel_ms": {k: round(v, 3) for k, v in splits.get(name, {}).items()}}
    del ws, wd, js, jd
    torch.cuda.empty_cache()
    out["note"] = ("median of 3 runs; select runs in place on a fresh copy each time; join rows/s "
                   "counts both input tables, as the paper does")
    return out


def run_to_table(args, g, stream, peak, peak_kind) -> dict:
    """Edge table (out-CSR order) and node table of the graph of the workload,
    timed with CUDA events over 5 launches after 2 warm-ups."""
    from paper_1503_07881_gb300 import ringo
    V, E = g.num_nodes, g.num_edges
    cols = (torch.empty(max(E, 1), dtype=torch.int32, device="cuda"),
            torch.empty(max(E, 1), dtype=torch.int32, device="cuda"))
    k = 5
    for _ in range(2):
        g.to_edge_table(ringo.RINGO_OUT, out=cols)
        g.to_node_table()
    torch.cuda.synchronize()
    ringo.ringo_profile_start()
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record(stream)
    for _ in range(k):
        g.to_edge_table(ringo.RINGO_OUT, out=cols)
    b.record(stream)
    for _ in range(k):
        g.to_node_table()
    c.record(stream)
    torch.cuda.synchronize()
    prof = {p["name"]: p for p in ringo.ringo_profile_stop()}
    edge_ms = a.elapsed_time(b) / k
    node_ms = b.elapsed_time(c) / k
    kern_ms = prof["edge_table"]["total_ms"] / k if "edge_table" in prof else edge_ms
    # per launch: neighbours read, one node-ID read per row end, two columns
    # written, the offsets and node IDs read once
    algo = 4 * E + 4 * E + 8 * E + 8 * (V + 1) + 4 * V
    del cols
    torch.cuda.empty_cache()
    rate = E / (edge_ms / 1e3)
    paper = PAPER_TO_TABLE_RATE.get(args.workload)
    return {"metric": "graph->table edges/s", "value": rate, "unit": "edges/s",
            "edge_table_ms": round(edge_ms, 3), "node_table_ms": round(node_ms, 3),
            "edges": E, "nodes": V, "paper_rate": paper,
            "vs_paper": rate / paper if paper else None,
            "roofline": {"bound": "hbm", "kernel": "k_expand", "achieved": algo / (kern_ms / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s",
                         "frac": algo / (kern_ms / 1e3) / 1e9 / peak,
                         "algorithmic_bytes": "16 B per edge + 12 B per node",
                         "peak_source": peak_kind}}


# ------------------------------------------------------ batched / served --
BATCH_PREDS, BATCH_LO, BATCH_HI = 4096, 1_000, 4_000_000
SERVE_LO, SERVE_HI, SERVE_TOPK, SERVE_BUDGET = 10_000, 50_000_000, 100, 120 << 30


def base_spec(scale: float = 1.0):
    """The base table of configs 4-5 (200M rows, 16M IDs, 10K tags), or a
    proportionally smaller one (profiling captures use scale 0.1)."""
    from paper_1503_07881_gb300 import tablegen
    full = tablegen.BaseSpec()
    if scale == 1.0:
        return full
    return tablegen.BaseSpec(rows=max(1, int(full.rows * scale)),
                             nodes=max(2, int(full.nodes * scale)),
                             tags=max(10, int(full.tags * scale)))


def load_base(seed: int, scale: float = 1.0):
    """The base table, generated on the device and loaded (clustered)."""
    from paper_1503_07881_gb300 import ringo, tablegen
    spec = base_spec(scale)
    cols = tablegen.make_base_table(spec, seed=seed, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    base = ringo.BaseTable(*cols)
    load_ms = (time.perf_counter() - t0) * 1e3
    del cols
    torch.cuda.empty_cache()
    return spec, base, load_ms


def plain_convert(ringo, base, pred, count: int, topk: int = 0):
    """One selection converted by the plain single-table calls (the loop the
    batched and served forms are compared with)."""
    src, dst = base.select_gather(pred, cap=max(1, count))
    g = ringo.ringo_table_to_graph(src, dst)
    if topk:
        g.degree_topk(0, topk)
        g.degree_topk(1, topk)
    g.free()


def run_batched(args, spec, base, steps: int, warmup: int) -> dict:
    from paper_1503_07881_gb300 import ringo, tablegen
    hi = max(BATCH_LO + 1, int(BATCH_HI * args.base_scale))
    preds = tablegen.make_predicates(spec, args.predicates, BATCH_LO, hi, seed=args.seed)
    counts = base.select_count(preds)
    R = int(counts.sum())
    peak, peak_kind = measured_peak_hbm()
    stream = torch.cuda.current_stream()
    info = None
    for _ in range(max(1, warmup)):
        bt = base.convert_batch(preds)
        if info is None:
            info = [bt.info(i) for i in range(len(preds))]
        bt.free()
    V = np.array([x["num_nodes"] for x in info], np.float64)
    E = np.array([x["num_edges"] for x in info], np.float64)
    N = counts.astype(np.float64)
    b0 = float((8 * N + 20 * V + 16 * (N > 0) + 8 * E).sum())
    bmodel = b0 + float((104 * N + 64 * E).sum())
    torch.cuda.synchronize()
    ringo.ringo_profile_start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        base.convert_batch(preds).free()
    end.record(stream)
    torch.cuda.synchronize()
    prof = ringo.ringo_profile_stop()
    ms = start.elapsed_time(end) / steps
    waves = sum(p["launches"] for p in prof if p["name"] == "batch_wave") // steps
    if args.no_plain:
        return {"workload": WORKLOADS["batched"], "predicates": len(preds), "selected_rows": R,
                "ms_per_step": round(ms, 3), "value": R / (ms / 1e3), "unit": "edges/s",
                "waves_per_step": waves}
    # the plain loop: select, gather and convert each table on its own
    for i in range(min(64, len(preds))):
        plain_convert(ringo, base, preds[i], int(counts[i]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, p in enumerate(preds):
        plain_convert(ringo, base, p, int(counts[i]))
    torch.cuda.synchronize()
    plain_ms = (time.perf_counter() - t0) * 1e3
    return {
        "workload": WORKLOADS["batched"], "predicates": len(preds), "selected_rows": R,
        "base_rows": spec.rows, "base_load_ms": None, "steps": steps,
        "ms_per_step": round(ms, 3), "value": R / (ms / 1e3), "unit": "edges/s",
        "waves_per_step": waves, "graphs_per_wave_launch": "one CUDA graph per wave",
        "b0_frac": b0 / (ms / 1e3) / 1e9 / peak, "model_frac": bmodel / (ms / 1e3) / 1e9 / peak,
        "peak_gbs": peak, "peak_source": peak_kind,
        "plain_loop": {"ms": round(plain_ms, 1), "value": R / (plain_ms / 1e3),
                       "unit": "edges/s",
                       "calls": "select_count + select_gather + ringo_table_to_graph per table"},
        "speedup_vs_plain": plain_ms / ms,
    }


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return t[t < duration]


def serve_with_server(ringo, base, preds, arrivals, workers: int, small_rows: int = 0) -> dict:
    import threading
    srv = ringo.Server(base, SERVE_BUDGET, workers=workers, small_rows=small_rows)
    tickets = [None] * len(preds)
    results = [None] * len(preds)
    t0 = ringo.clock_ns() + 20_000_000

    def collect():
        for i in range(len(preds)):
            while tickets[i] is None:
                time.sleep(0.0002)
            results[i] = srv.wait(tickets[i])

    th = threading.Thread(target=collect)
    ringo.ringo_profile_start()
    th.start()
    for i, p in enumerate(preds):
        due = t0 + int(arrivals[i] * 1e9)
        while True:
            dt = due - ringo.clock_ns()
            if dt <= 0:
                break
            time.sleep(min(dt / 1e9, 0.001) if dt > 200_000 else 0)
        tickets[i] = srv.submit(p, topk=SERVE_TOPK)
    th.join()
    st = srv.stats()
    srv.close()
    prof = {p["name"]: {"n": p["launches"], "ms": round(p["total_ms"], 2)}
            for p in ringo.ringo_profile_stop()
            if p["name"].startswith("host:") or p["name"] == "batch_wave"}
    lat = np.array([(r["t_done_ns"] - (t0 + int(a * 1e9))) / 1e6 for r, a in zip(results, arrivals)])
    rows = sum(r["nrows"] for r in results)
    span = (max(r["t_done_ns"] for r in results) - t0) / 1e9
    bad = sum(r["status"] != 0 for r in results)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "edges_per_s": rows / span, "failed": bad,
            "batches": st["batches"], "mean_batch": len(preds) / max(1, st["batches"]),
            "max_concurrent_batches": st["max_concurrent_batches"],
            "max_inflight_gb": st["max_inflight_bytes"] / 1e9, "time_split": prof}


def serve_plain(ringo, base, preds, arrivals, deadline_s: float) -> dict:
    """One request at a time in arrival order.  A loop that falls behind
    stops `deadline_s` after the first arrival: the requests it has not
    served by then count with their latency at that moment (a lower bound),
    and the result says it saturated."""
    counts = base.select_count(preds)
    t0 = ringo.clock_ns() + 20_000_000
    stop = t0 + int(deadline_s * 1e9)
    lat = []
    done_rows = 0
    for i, p in enumerate(preds):
        due = t0 + int(arrivals[i] * 1e9)
        while ringo.clock_ns() < due:
            time.sleep(0.0002)
        if ringo.clock_ns() >= stop:
            break
        plain_convert(ringo, base, p, int(counts[i]), SERVE_TOPK)
        lat.append((ringo.clock_ns() - due) / 1e6)
        done_rows += int(counts[i])
    end = ringo.clock_ns()
    served = len(lat)
    lat += [(end - (t0 + int(a * 1e9))) / 1e6 for a in arrivals[served:]]
    span = (end - t0) / 1e9
    lat = np.array(lat)
    out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "edges_per_s": done_rows / span,
           "served": served, "requests": len(preds)}
    if served < len(preds):
        out["saturated"] = True
        out["note"] = (f"stopped {deadline_s:.0f} s after the first arrival with {len(preds) - served} "
                       "requests unserved; their latency at that moment counts, so p50/p99 are "
                       "lower bounds")
    return out


def run_served(args, spec, base, rates, duration: float) -> dict:
    from paper_1503_07881_gb300 import ringo, tablegen
    out = []
    for k, rate in enumerate(rates):
        arr = poisson_arrivals(rate, duration, args.seed + k)
        preds = tablegen.make_predicates(spec, len(arr), SERVE_LO, SERVE_HI, seed=args.seed + 100 + k)
        warm = tablegen.make_predicates(spec, 8, SERVE_LO, SERVE_HI, seed=args.seed + 999)
        srv = ringo.Server(base, SERVE_BUDGET)
        for p in warm:
            srv.wait(srv.submit(p, topk=SERVE_TOPK))
        srv.close()
        gc.disable()  # no collector pauses in the client's submit loop
        try:
            server = serve_with_server(ringo, base, preds, arr, workers=args.serve_workers,
                                       small_rows=args.serve_small_rows)
        finally:
            gc.enable()
        row = {"rate_per_s": rate, "duration_s": duration, "requests": len(preds),
               "workers": args.serve_workers,
               "small_lane_rows": (1 << 21) if args.serve_small_rows == 0 else args.serve_small_rows,
               "server": server}
        if not args.no_plain:
            gc.disable()
            try:
                plain = serve_plain(ringo, base, preds, arr, deadline_s=2 * duration + 2)
            finally:
                gc.enable()
            row["plain_loop"] = plain
            row["p99_speedup_vs_plain"] = plain["p99_ms"] / server["p99_ms"]
        out.append(row)
    return {"workload": WORKLOADS["served"], "budget_bytes": SERVE_BUDGET, "topk": SERVE_TOPK,
            "latency": "scheduled arrival to result ready (no coordinated omission)",
            "rates": out}


def run_base_workloads(args) -> tuple[dict | None, dict | None]:
    """Batched and served runs on the resident base table."""
    batched = served = None
    only = args.workload in ("batched", "served")
    do_batched = args.workload == "batched" or (not only and not args.no_batched)
    do_served = args.workload == "served" or (not only and not args.no_served)
    spec, base, load_ms = load_base(args.seed, args.base_scale)
    try:
        if do_batched:
            try:
                batched = run_batched(args, spec, base, steps=args.batch_steps, warmup=1)
                batched["base_load_ms"] = round(load_ms, 1)
            except Exception as e:  # reported, not fatal to the plain line
                batched = {"error": f"{type(e).__name__}: {e}"}
        if do_served:
            try:
                served = run_served(args, spec, base, args.serve_rates, args.serve_seconds)
            except Exception as e:
                served = {"error": f"{type(e).__name__}: {e}"}
    finally:
        base.free()
        torch.cuda.empty_cache()
    return batched, served


# ------------------------------------------------------- reference arm ----
def run_reference(args, rank):
    """The oracle, as it stands, on bounded samples of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_1503_07881_gb300 import tablegen

    if args.workload in ("batched", "served"):
        return run_reference_base(args)
    spec = tablegen.SPECS[args.workload]
    S = min(spec.rows, REF_SAMPLE_ROWS[args.workload])
    n_slices = args.warmup + args.steps
    slices = []
    for k in range(n_slices):
        lo = (k * S) % max(1, spec.rows - S + 1)
        s, d = tablegen.make_table(spec, seed=args.seed, device="cpu", start=lo, count=S)
        slices.append((s.numpy(), d.numpy()))
    for k in range(args.warmup):
        oracle.table_to_graph(*slices[k])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.table_to_graph(*slices[args.warmup + k])
    dt = time.perf_counter() - t0
    ms = dt * 1e3 / args.steps
    value = S / (ms / 1e3)
    line = {
        "impl": "reference",
        "metric": "table->graph edges/s",
        "value": value,
        "unit": "edges/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (value / PAPER_RATE[args.workload]) if args.workload in PAPER_RATE else None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "rows_per_step": S,
                   "note": "each step converts a different bounded slice of the workload"},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"{S}-row slices of the workload, one per step"},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_base(args):
    """The oracle on the selections of a bounded base table of the same shape
    (1M rows, 10K Zipf tags, five years of timestamps): each step converts
    the next batch of selections, host-side select included."""
    import oracle
    from paper_1503_07881_gb300 import tablegen

    spec = tablegen.BaseSpec(rows=1_000_000, nodes=80_000, tags=10_000)
    src, dst, ts, tag = (c.numpy() for c in tablegen.make_base_table(spec, seed=args.seed))
    lo, hi = (BATCH_LO, BATCH_HI) if args.workload == "batched" else (SERVE_LO, SERVE_HI)
    scale = spec.rows / tablegen.BaseSpec().rows
    preds = tablegen.make_predicates(spec, 64 * (args.warmup + args.steps),
                                     max(1, int(lo * scale)), max(2, int(hi * scale)),
                                     seed=args.seed)

    def step(ps):
        rows = 0
        for tags, t0, t1 in ps:
            m = np.isin(tag, np.asarray(tags, np.int32)) & (ts >= t0) & (ts < t1)
            oracle.table_to_graph(src[m], dst[m])
            rows += int(m.sum())
        return rows

    for k in range(args.warmup):
        step(preds[64 * k:64 * (k + 1)])
    t0 = time.perf_counter()
    rows = 0
    for k in range(args.warmup, args.warmup + args.steps):
        rows += step(preds[64 * k:64 * (k + 1)])
    dt = time.perf_counter() - t0
    value = rows / dt
    line = {"impl": "reference", "metric": f"table->graph edges/s, {args.workload}",
            "value": value, "unit": "edges/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "note": "64 selections per step from a 1M-row base table of the same shape"},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": "64 selections per step, sizes scaled by 1/200"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="twitter")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched summary")
    ap.add_argument("--no-to-table", action="store_true", help="skip the graph->table summary")
    ap.add_argument("--no-served", action="store_true", help="skip the served summary")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain per-table / per-request loops (profiling, sweeps)")
    ap.add_argument("--base-scale", type=float, default=1.0,
                    help="scale of the base table and of the largest selection (profiling)")
    ap.add_argument("--predicates", type=int, default=BATCH_PREDS)
    ap.add_argument("--serve-rates", type=lambda x: [float(v) for v in x.split(",")],
                    default=[100.0, 200.0, 500.0, 1000.0, 2000.0])
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-workers", type=int, default=1, help="server worker threads (streams)")
    ap.add_argument("--serve-small-rows", type=int, default=0,
                    help="small-request lane threshold in rows (0: 2^21, -1: no small lane)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("note: fewer than 3 warm-up steps requested; using 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup(args)
    try:
        if args.workload in ("batched", "served"):
            if rank == 0:
                run_base_only(args)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
