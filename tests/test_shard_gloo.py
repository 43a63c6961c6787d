"""Host-side multi-rank logic on CPU (gloo, world size 2): query sharding is a
disjoint, complete, balanced partition identical on every rank, and the
benchmark's reduction takes the max of the times and the sum of the checks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2411_13507_gb300 import shard
from paper_2411_13507_gb300 import synth


def test_lpt_partition_is_complete_and_balanced():
    probs = synth.batched_queries(seed=3, Q=64, n_lo=100, n_hi=4000, k_lo=4, k_hi=32, t_lo=4, t_hi=16)
    work = [shard.estimate_work(p.N, p.K, p.nT) for p in probs]
    for world in (1, 2, 3, 8):
        parts = shard.shard_queries(work, world)
        flat = sorted(q for part in parts for q in part)
        assert flat == list(range(len(work)))
        loads = [sum(work[q] for q in part) for part in parts]
        # LPT bound: max load <= mean + max single job
        assert max(loads) <= sum(work) / world + max(work) + 1e-9
    with pytest.raises(ValueError):
        shard.shard_queries(work, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = [float(1 + (i * 37) % 11) for i in range(20)]
        parts = shard.shard_queries(work, world)
        mine = parts[rank]
        checks = sum(work[i] for i in mine)
        times = [0.5 + rank, 2.0 - rank]
        t, c = shard.aggregate(times, checks, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, parts)
        q.put((rank, t, c, gathered, mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    work_total = sum(float(1 + (i * 37) % 11) for i in range(20))
    for rank, t, c, gathered, mine in res:
        assert t == [1.5, 2.0]                      # max over ranks, per entry
        assert c == pytest.approx(work_total)       # sum of the ranks' checks
        assert gathered[0] == gathered[1]           # every rank computed the same partition
    assert sorted(res[0][4] + res[1][4]) == list(range(20))
