"""Multi-GPU placement of the edge build.

Independent queries (replicas, weak scaling): the edge build of one query
never needs data from another, so N GPUs run as N replicas -- queries are
dealt to ranks by a greedy longest-processing-time rule on an estimated work
(candidate checks ~ sum_k n_k^2 * nT, approximated from N^2 / K * nT), every
rank builds and searches its own queries, and the only communication is the
timing/throughput reduction of the benchmark.  No collective touches the data
path.

One query over several GPUs (buildGraph of Algorithm 1 at a size one GPU
would split): rank r builds the source rows of shard r of the world
(plan_build_edges_shard: contiguous row ranges of equal pair-slot work, cut
identically on every rank from the same membership), so each rank's rows are
final and the ranks' rows follow one another in rank order.  One exchange
step then gives every rank the whole graph for its search replica: an
all-gather of (edge count, row range) per rank, then an all-gather of one
byte payload per rank (padded to the largest) holding its rows' offsets and
its edges' columns, weights, masks and duration indices.  The merge
concatenates the pieces in rank order and shifts each rank's row offsets by
the edges of the ranks before it; no arithmetic of the method is involved,
and the result equals the single-GPU graph bit for bit.
"""
from __future__ import annotations

import heapq
from typing import List, Optional, Sequence


def estimate_work(N: int, K: int, nT: int) -> float:
    """Rough cost of a query: expected candidate pairs (N^2/K) times durations."""
    return float(N) * float(N) / max(1, K) * max(1, nT)


def shard_queries(work: Sequence[float], world: int) -> List[List[int]]:
    """Greedy LPT: queries in decreasing work, each to the least-loaded rank.
    Returns, per rank, the ascending list of query indices it owns."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [(0.0, r) for r in range(world)]
    heapq.heapify(loads)
    owned: List[List[int]] = [[] for _ in range(world)]
    for q in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        load, r = heapq.heappop(loads)
        owned[r].append(q)
        heapq.heappush(loads, (load + float(work[q]), r))
    return [sorted(o) for o in owned]


def aggregate(times_s: Sequence[float], checks: float, dist=None, device=None):
    """Whole-job throughput inputs: the max over ranks of each time and the sum of
    the checks.  With dist=None (one process) the values are returned as is."""
    if dist is None:
        return list(times_s), float(checks)
    import torch
    t = torch.tensor(list(times_s), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(checks)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), float(c.item())


def row_split(row_work: Sequence[int], nshard: int) -> List[tuple]:
    """The cut rule of plan_build_edges_shard: with S_i the work of rows < i and
    W the total, shard r starts at the number of rows with S_i * nshard < W * r;
    the last shard ends at the last row.  Returns [(lo, hi)] per shard."""
    import numpy as np
    w = np.asarray(row_work, dtype=np.int64)
    N = int(w.shape[0])
    S = np.concatenate([[0], np.cumsum(w)[:-1]]) if N else np.zeros(0, np.int64)
    W = int(w.sum())
    bounds = [int(np.count_nonzero(S * nshard < W * r)) for r in range(nshard)] + [N]
    return [(bounds[r], bounds[r + 1]) for r in range(nshard)]


def _bytes(t):
    import torch
    return t.contiguous().view(torch.uint8)


def pack(row_off, col, w, mask, tidx, E: int, lo: int, hi: int, nbytes: Optional[int] = None):
    """One rank's payload: w | row offsets of rows lo+1..hi | col | mask | tidx
    (weights first, so every segment starts at a multiple of its element size),
    zero-padded to nbytes."""
    import torch
    parts = [_bytes(w[:E]), _bytes(row_off[lo + 1:hi + 1]), _bytes(col[:E]), _bytes(mask[:E]), _bytes(tidx[:E])]
    n = sum(int(p.numel()) for p in parts)
    size = n if nbytes is None else int(nbytes)
    out = torch.zeros(size, dtype=torch.uint8, device=col.device)
    o = 0
    for p in parts:
        out[o:o + p.numel()] = p
        o += int(p.numel())
    return out


def payload_bytes(E: int, lo: int, hi: int, wsize: int) -> int:
    return E * (wsize + 4 + 4 + 1) + (hi - lo) * 4


def unpack(buf, E: int, lo: int, hi: int, wdtype) -> dict:
    import torch
    ws = torch.empty(0, dtype=wdtype).element_size()
    o = 0
    out = {}
    for key, n, dt in (("w", E * ws, wdtype), ("rows", (hi - lo) * 4, torch.int32), ("col", E * 4, torch.int32),
                       ("mask", E * 4, torch.int32), ("tidx", E, torch.uint8)):
        out[key] = buf[o:o + n].view(dt)
        o += n
    return out


def merge(pieces: Sequence[dict], ranges: Sequence[tuple], counts: Sequence[int], N: int) -> dict:
    """The whole graph from the shards' pieces (in rank order)."""
    import torch
    assert ranges[0][0] == 0 and ranges[-1][1] == N and all(ranges[r][1] == ranges[r + 1][0]
                                                            for r in range(len(ranges) - 1)), "shards must tile the rows"
    dev = pieces[0]["col"].device
    row_off = torch.zeros(N + 1, dtype=torch.int32, device=dev)
    base = 0
    for (lo, hi), E, pc in zip(ranges, counts, pieces):
        row_off[lo + 1:hi + 1] = pc["rows"] + base
        base += int(E)
    return {"row_off": row_off, "col": torch.cat([p["col"] for p in pieces]),
            "w": torch.cat([p["w"] for p in pieces]), "mask": torch.cat([p["mask"] for p in pieces]),
            "tidx": torch.cat([p["tidx"] for p in pieces]), "count": base}


def exchange(row_off, col, w, mask, tidx, E: int, lo: int, hi: int, N: int, dist, group=None) -> dict:
    """All-gather-v of the shards' CSR pieces (counts and row ranges first, then
    the padded payload); every rank returns the whole graph (merge)."""
    import torch
    dev = col.device
    world = dist.get_world_size(group)
    head = torch.tensor([E, lo, hi], dtype=torch.int64, device=dev)
    heads = [torch.empty_like(head) for _ in range(world)]
    dist.all_gather(heads, head, group=group)
    hv = [tuple(int(x) for x in h.tolist()) for h in heads]
    ws = w.element_size()
    nbytes = max(payload_bytes(e, a, b, ws) for e, a, b in hv)
    nbytes = (nbytes + 15) // 16 * 16
    buf = pack(row_off, col, w, mask, tidx, E, lo, hi, nbytes)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    pieces = [unpack(b, e, a, c, w.dtype) for b, (e, a, c) in zip(bufs, hv)]
    return merge(pieces, [(a, c) for _, a, c in hv], [e for e, _, _ in hv], N)
