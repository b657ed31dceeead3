"""Full-size checks of a GPU result that need no oracle run over the whole
table: structural properties computed with plain torch ops on the device, and
exact neighbour lists of sampled nodes from the oracle's one-pass scan."""
from __future__ import annotations

import numpy as np
import torch

import oracle


def graph_arrays(g) -> dict:
    off_o, nbr_o = g.csr(0)
    off_i, nbr_i = g.csr(1)
    return {"node_ids": g.node_ids(), "out_off": off_o, "out_nbr": nbr_o,
            "in_off": off_i, "in_nbr": nbr_i, "num_nodes": g.num_nodes,
            "num_edges": g.num_edges}


def _owners(off: torch.Tensor, E: int) -> torch.Tensor:
    deg = off[1:] - off[:-1]
    return torch.repeat_interleave(torch.arange(deg.numel(), device=off.device), deg,
                                   output_size=E)


def check_properties(a: dict, src: torch.Tensor, dst: torch.Tensor) -> None:
    """Invariants of the definition (paper Section 3.4 / 3.2) at any size."""
    ids = a["node_ids"].long()
    V, E = a["num_nodes"], a["num_edges"]
    assert ids.numel() == V
    if V > 1:
        assert bool((ids[1:] > ids[:-1]).all()), "node_ids not strictly increasing"
    keys = {}
    for d in ("out", "in"):
        off, nbr = a[f"{d}_off"], a[f"{d}_nbr"].long()
        assert off.numel() == V + 1 and int(off[0]) == 0 and int(off[-1]) == E
        assert bool((off[1:] >= off[:-1]).all())
        if E:
            assert int(nbr.min()) >= 0 and int(nbr.max()) < V
            own = _owners(off, E)
            k = own * V + nbr
            assert bool((k[1:] > k[:-1]).all()), f"{d} lists not strictly increasing"
            keys[d] = k
            del own
    # every node has at least one edge
    deg = (a["out_off"][1:] - a["out_off"][:-1]) + (a["in_off"][1:] - a["in_off"][:-1])
    assert V == 0 or int(deg.min()) >= 1
    if E == 0:
        assert src.numel() == 0
        return
    # v in out(u) iff u in in(v): transposed in-keys are exactly the out-keys
    ki = keys["in"]
    t = (ki % V) * V + torch.div(ki, V, rounding_mode="floor")
    t, _ = torch.sort(t)
    assert torch.equal(t, keys["out"]), "in-CSR is not the transpose of out-CSR"
    del t, ki
    # every row is an edge, and every edge is a row
    rs = torch.searchsorted(ids, src.long())
    rd = torch.searchsorted(ids, dst.long())
    assert int(rs.max()) < V and int(rd.max()) < V
    assert torch.equal(ids[rs], src.long()) and torch.equal(ids[rd], dst.long()), \
        "a column value is missing from node_ids"
    rk = rs * V + rd
    del rs, rd
    pos = torch.searchsorted(keys["out"], rk)
    assert int(pos.max()) < E and torch.equal(keys["out"][pos], rk), "a row has no edge"
    del pos
    uniq = torch.unique(rk)
    assert uniq.numel() == E, "E differs from the number of distinct rows"


def check_samples(a: dict, src_h: np.ndarray, dst_h: np.ndarray, sample_ids: np.ndarray) -> None:
    """Exact out/in lists of sampled node IDs against the oracle's scan."""
    outs, ins, present = oracle.sample_lists(src_h, dst_h, sample_ids)
    ids = a["node_ids"].cpu().numpy()
    oo, on = a["out_off"].cpu().numpy(), a["out_nbr"]
    io, inn = a["in_off"].cpu().numpy(), a["in_nbr"]
    for k, x in enumerate(sample_ids):
        r = int(np.searchsorted(ids, x))
        found = r < ids.size and ids[r] == x
        assert found == bool(present[k]), f"node {x}: presence differs"
        if not found:
            continue
        got_o = ids[on[oo[r]:oo[r + 1]].cpu().numpy()]
        got_i = ids[inn[io[r]:io[r + 1]].cpu().numpy()]
        assert np.array_equal(got_o, outs[k]), f"out-list of node {x} differs"
        assert np.array_equal(got_i, ins[k]), f"in-list of node {x} differs"


def pick_samples(src_h: np.ndarray, dst_h: np.ndarray, ids: np.ndarray, a: dict,
                 n_random: int = 200, seed: int = 0) -> np.ndarray:
    """Random nodes, the top out- and in-degree nodes, the extremes, and IDs
    that are not nodes."""
    rng = np.random.default_rng(seed)
    pick = [ids[rng.integers(0, ids.size, n_random)], ids[:3], ids[-3:]]
    for d in ("out", "in"):
        off = a[f"{d}_off"]
        deg = off[1:] - off[:-1]
        top = torch.topk(deg, min(5, deg.numel())).indices.cpu().numpy()
        pick.append(ids[top])
    absent = np.array([-7, 2**31 - 3, -(2**31) + 5], np.int64)
    absent = absent[~np.isin(absent, ids)].astype(np.int32)
    pick.append(absent)
    return np.unique(np.concatenate(pick).astype(np.int32))


def check_undirected(u: dict, d: dict, chunk: int = 1 << 30) -> None:
    """The undirected graph u of a table against the directed graph d of the
    same table (whose own invariants check_properties establishes): the same
    node list, both CSRs of u equal, and every node's list the sorted union of
    its out- and in-lists in d.  Node ranges of at most `chunk` entries at a
    time, so no torch operation sees more than 2^31 elements."""
    V = d["num_nodes"]
    assert u["num_nodes"] == V and torch.equal(u["node_ids"], d["node_ids"])
    assert torch.equal(u["out_off"], u["in_off"]) and torch.equal(u["out_nbr"], u["in_nbr"])
    uo, oo, io = u["out_off"], d["out_off"], d["in_off"]
    assert uo.numel() == V + 1 and int(uo[0]) == 0 and int(uo[-1]) == u["num_edges"]
    w = oo + io  # merged positions before each node
    v0 = 0
    while v0 < V:
        v1 = int(torch.searchsorted(w, w[v0] + chunk, right=True)) - 1
        v1 = min(max(v1, v0 + 1), V)
        nodes = torch.arange(v1 - v0, device=uo.device)

        def keys(off, nbr):
            deg = off[v0 + 1:v1 + 1] - off[v0:v1]
            own = torch.repeat_interleave(nodes, deg, output_size=int(deg.sum()))
            return own * V + nbr[int(off[v0]):int(off[v1])].long()

        want = torch.unique(torch.cat([keys(oo, d["out_nbr"]), keys(io, d["in_nbr"])]))
        got = keys(uo, u["out_nbr"])
        assert torch.equal(got, want), f"lists of nodes {v0}..{v1 - 1} differ"
        del want, got
        v0 = v1


def check_undirected_samples(a: dict, src_h: np.ndarray, dst_h: np.ndarray,
                             sample_ids: np.ndarray) -> None:
    """The lists of sampled node IDs against the oracle's one-pass scan: the
    neighbours of x are the union of its out- and in-neighbours."""
    outs, ins, present = oracle.sample_lists(src_h, dst_h, sample_ids)
    ids = a["node_ids"].cpu().numpy()
    off, nbr = a["out_off"].cpu().numpy(), a["out_nbr"]
    for k, x in enumerate(sample_ids):
        r = int(np.searchsorted(ids, x))
        found = r < ids.size and ids[r] == x
        assert found == bool(present[k]), f"node {x}: presence differs"
        if found:
            got = ids[nbr[off[r]:off[r + 1]].cpu().numpy()]
            assert np.array_equal(got, np.union1d(outs[k], ins[k])), f"list of node {x} differs"
