"""Multi-GPU placement of independent planning queries (replicas, weak scaling).

The edge build of one query never needs data from another, so N GPUs run as N
replicas: queries are dealt to ranks by a greedy longest-processing-time rule
on an estimated work (candidate checks ~ sum_k n_k^2 * nT, approximated from
N^2 / K * nT), every rank builds and searches its own queries, and the only
communication is the timing/throughput reduction of the benchmark (max of the
per-rank times, sum of the per-rank checks).  No collective touches the data
path.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


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
