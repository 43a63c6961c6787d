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


# ---------------------------------------------------------------------------
# One query over several ranks: each rank's rows (the equal-work row split),
# then the all-gather-v exchange of the CSR pieces; every rank must end with
# the single-rank graph, bit for bit.  The rank's piece here is the oracle's
# FP64 CSR restricted to its rows (the GPU builds the same rows with
# plan_build_edges_shard, tested on the GPU).
# ---------------------------------------------------------------------------
def _row_work(op):
    inm = op.membership().astype(bool)           # [N][K]
    nk = inm.sum(axis=0).astype("int64")
    return (inm * nk[None, :]).sum(axis=1)


def _oracle_piece(op, lo, hi):
    import numpy as np
    rows = np.arange(lo, hi, dtype=np.int32)
    e = op.edges(rows, with_detail=False)
    keep = e["mask"] != 0
    i = e["i"][keep].astype(np.int64)
    row_off = np.zeros(op.N + 1, dtype=np.int64)
    np.add.at(row_off, i + 1, 1)
    row_off = np.cumsum(row_off)
    return {"row_off": torch.as_tensor(row_off.astype(np.int32)), "col": torch.as_tensor(e["j"][keep]),
            "w": torch.as_tensor(e["w"][keep]), "mask": torch.as_tensor(e["mask"][keep].view(np.int32)),
            "tidx": torch.as_tensor(e["t"][keep].astype(np.uint8)), "E": int(keep.sum())}


def _shard_worker(rank, world, port, q):
    import numpy as np
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = synth.double_integrator_2d(seed=4, N=300, K=8, nT=6)
        op = oracle.OracleProblem(prob)
        ranges = shard.row_split(_row_work(op), world)
        lo, hi = ranges[rank]
        pc = _oracle_piece(op, lo, hi)
        g = shard.exchange(pc["row_off"], pc["col"], pc["w"], pc["mask"], pc["tidx"], pc["E"], lo, hi, op.N, dist)
        full = op.csr()
        ok = (np.array_equal(g["row_off"].numpy(), full["row_off"]) and np.array_equal(g["col"].numpy(), full["col"])
              and np.array_equal(g["w"].numpy(), full["w"])
              and np.array_equal(g["mask"].numpy().view(np.uint32), full["mask"])
              and np.array_equal(g["tidx"].numpy().astype(np.int32), full["t"]) and g["count"] == len(full["col"]))
        q.put((rank, bool(ok), (lo, hi), pc["E"], g["count"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_shards_exchange_to_the_single_rank_graph_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _, _ in res), res
    ranges = [r[2] for r in res]
    assert ranges[0][0] == 0 and all(ranges[k][1] == ranges[k + 1][0] for k in range(world - 1))
    assert sum(r[3] for r in res) == res[0][4]     # the pieces add up to the whole graph
    assert min(r[3] for r in res) > 0              # every rank built part of it


def test_row_split_rule():
    """Equal-work contiguous cuts: complete, ordered, and each shard's work within one row of W / nshard."""
    import numpy as np
    rng = np.random.default_rng(2)
    for trial in range(20):
        w = rng.integers(0, 50, size=int(rng.integers(1, 400)))
        w[rng.random(w.shape[0]) < 0.2] = 0
        for ns in (1, 2, 3, 7):
            rs = shard.row_split(w, ns)
            assert rs[0][0] == 0 and rs[-1][1] == w.shape[0]
            assert all(rs[k][1] == rs[k + 1][0] for k in range(ns - 1))
            W = int(w.sum())
            for lo, hi in rs:
                assert int(w[lo:hi].sum()) <= W / ns + (w.max() if w.size else 0) + 1e-9
    assert shard.row_split([0, 0, 0], 2) == [(0, 0), (0, 3)]
