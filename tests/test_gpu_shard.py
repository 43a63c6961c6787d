"""One query's edge build split over shards of source rows
(plan_build_edges_shard), the multi-GPU form of buildGraph (Algorithm 1):
every shard is built here on the one GPU, one after the other, and merged by
the same pack / unpack / merge code that the all-gather-v exchange runs
between ranks.  Bar: the device's row ranges equal the cut rule applied to the
oracle's membership; the merged graph equals the single build bit for bit
(row offsets, columns, masks, weights, duration indices) and the oracle
(tests/parity.py); the shards' candidate counts add up to the single build's.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import shard, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def row_work(op):
    inm = op.membership().astype(bool)
    nk = inm.sum(axis=0).astype(np.int64)
    return (inm * nk[None, :]).sum(axis=1)


def build_sharded(pl, dp, nshard):
    pieces, ranges, counts, cand = [], [], [], 0
    for r in range(nshard):
        g = pl.build_edges_shard(dp, r, nshard)
        info = pl.info()
        lo, hi = int(info["shard_lo"]), int(info["shard_hi"])
        E = g.E
        buf = shard.pack(g.row_off, g.col, g.w, g.mask, g.tidx, E, lo, hi)
        pieces.append(shard.unpack(buf, E, lo, hi, g.w.dtype))
        ranges.append((lo, hi))
        counts.append(E)
        cand += int(info["candidates"])
        # rows outside the shard are empty
        ro = g.row_off.cpu().numpy()
        assert np.all(ro[:lo + 1] == 0) and np.all(ro[hi:] == E)
    return shard.merge(pieces, ranges, counts, dp.N), ranges, cand


def same(merged, single):
    E = single.E
    assert merged["count"] == E
    assert torch.equal(merged["row_off"], single.row_off)
    for k in ("col", "w", "mask", "tidx"):
        assert torch.equal(merged[k], getattr(single, k)[:E]), k


@pytest.mark.parametrize("case", ["f32-3d", "f64-2d"])
def test_row_shards_merge_to_the_single_build(case):
    if case == "f32-3d":
        prob = synth.triple_integrator_3d(seed=1, N=2048, K=16)
        arith, inp = "f32", "f32"
    else:
        prob = synth.double_integrator_2d(seed=2)
        arith, inp = "f64", "f64"
    pl = P.Planner.for_problem(prob, arith=arith, input=inp)
    dp = P.to_device(prob, input=inp)
    single = pl.build_edges(dp)
    cand = int(pl.info()["candidates"])
    op = oracle.OracleProblem(prob)
    work = row_work(op)
    csr = op.csr(with_detail=True)
    for nshard in (1, 2, 3, 5):
        merged, ranges, c = build_sharded(pl, dp, nshard)
        assert ranges == shard.row_split(work, nshard), (nshard, ranges)
        same(merged, single)
        assert c == cand
    g = {"row_off": merged["row_off"].cpu().numpy().astype(np.int64), "col": merged["col"].cpu().numpy(),
         "w": merged["w"].cpu().numpy().astype(np.float64), "t": merged["tidx"].cpu().numpy().astype(np.int32),
         "mask": merged["mask"].cpu().numpy().view(np.uint32)}
    parity.compare_full(g, csr, prob.N, prob.nT, arith)
    pl.close()


def test_more_shards_than_busy_rows_and_other_pipelines():
    """Shards with no rows, and every FP32 pair pipeline: the merged graph is unchanged."""
    prob = synth.triple_integrator_3d(seed=5, N=600, K=6, nT=8)
    pl = P.Planner.for_problem(prob, arith="f32", input="f32")
    dp = P.to_device(prob, input="f32")
    single = pl.build_edges(dp)
    for tile, chunks, pipe in ((0, 0, 0), (32, 3, 0), (64, 2, 1), (20, 4, 2)):
        pl.set_tile(tile, 0, chunks, pipe)
        for nshard in (4, 64):
            merged, ranges, _ = build_sharded(pl, dp, nshard)
            same(merged, single)
    pl.close()


def test_precision_form_shards():
    prob = synth.double_integrator_2d(seed=1, N=256, K=8)
    for arith in ("tf32", "bf16"):
        pl = P.Planner.for_problem(prob, arith=arith, input="f64")
        dp = P.to_device(prob, input="f64")
        single = pl.build_edges(dp)
        merged, _, _ = build_sharded(pl, dp, 3)
        same(merged, single)
        pl.close()


def test_row_shards_at_the_benchmark_size():
    """The 3-D benchmark workload (N = 8192, K = 64, nT = 16) in four shards:
    the merged graph equals the single build bit for bit, and the shards'
    work is balanced (each within 5% of a quarter of the candidates)."""
    prob = synth.triple_integrator_3d(seed=2)
    pl = P.Planner.for_problem(prob, arith="f32", input="f32")
    dp = P.to_device(prob, input="f32")
    single = pl.build_edges(dp)
    cand = int(pl.info()["candidates"])
    per = []
    for r in range(4):
        pl.build_edges_shard(dp, r, 4)
        per.append(int(pl.info()["candidates"]))
    merged, ranges, c = build_sharded(pl, dp, 4)
    same(merged, single)
    assert c == cand and sum(per) == cand
    assert max(per) <= 1.05 * cand / 4, per
    pl.close()
