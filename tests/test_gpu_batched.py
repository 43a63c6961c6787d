"""Batching form on the GPU: many uneven queries in one pass (one persistent
pair launch), captured in a CUDA graph and replayed, with autotuned tiles.
Every query's graph must equal the single-query build bit for bit and the
oracle's (bar: tests/parity.py)."""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402
from paper_2411_13507_gb300 import autotune  # noqa: E402


def small_batch(seed=3, Q=7):
    return synth.batched_queries(seed=seed, Q=Q, n_lo=150, n_hi=900, k_lo=2, k_hi=12, t_lo=3, t_hi=9)


def same_graph(a: dict, b: dict):
    for k in ("row_off", "col", "mask", "t"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["w"], b["w"])


def test_batched_equals_single_and_oracle():
    probs = small_batch()
    pl = P.Planner.for_problem(probs[0], arith="f32", input="f32")
    dps = [P.to_device(p, input="f32") for p in probs]
    graphs = pl.build_batched(dps)
    info = pl.info()
    tot_cand = 0
    for q, (p, dp, g) in enumerate(zip(probs, dps, graphs)):
        single = P.Planner.for_problem(p, arith="f32", input="f32")
        gs = single.build_edges(dp)
        same_graph(g.to_numpy(), gs.to_numpy())
        tot_cand += single.info()["candidates"]
        if q < 3:
            csr = oracle.OracleProblem(p).csr(with_detail=True)
            parity.compare_full(g.to_numpy(), csr, p.N, p.nT, "f32")
    assert info["candidates"] == tot_cand


def test_batched_with_empty_and_fp64_queries():
    probs = small_batch(seed=5, Q=4)
    probs[1].states = probs[1].states[:0]            # N = 0
    probs[2].poly_off = probs[2].poly_off[:1]        # K = 0
    probs[2].A = probs[2].A[:0]
    probs[2].b = probs[2].b[:0]
    pl = P.Planner.for_problem(probs[0], arith="f32", input="f32")
    dps = [P.to_device(p, input="f32") for p in probs]
    graphs = pl.build_batched(dps)
    for p, g in zip(probs, graphs):
        csr = oracle.OracleProblem(p).csr(with_detail=True)
        parity.compare_full(g.to_numpy(), csr, p.N, p.nT, "f32")


def test_graph_capture_replay_follows_inputs():
    probs = small_batch(seed=7, Q=5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pl = P.Planner.for_problem(probs[0], arith="f32", input="f32", stream=stream)
        dps = [P.to_device(p, input="f32") for p in probs]
        graphs = pl.build_batched(dps, cap_per_state=1000)  # sizes scratch and outputs, prepares
        ref = [g.to_numpy() for g in graphs]
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            pl.build_batched_async()
        for g in graphs:
            g.count.zero_()
            g.col.zero_()
        cg.replay()
        stream.synchronize()
        assert pl.wait() == P.PLAN_OK
        for r, g in zip(ref, graphs):
            same_graph(g.to_numpy(), r)
        # move the states of query 0 in place: the replay must see the new inputs
        new = synth.batched_queries(seed=99, Q=1, n_lo=probs[0].N, n_hi=probs[0].N, k_lo=probs[0].K,
                                    k_hi=probs[0].K, t_lo=probs[0].nT, t_hi=probs[0].nT)[0]
        probs[0].states = new.states[:probs[0].N]
        dps[0].states.copy_(torch.as_tensor(probs[0].states, dtype=torch.float32))
        cg.replay()
        stream.synchronize()
        assert pl.wait() == P.PLAN_OK
        csr = oracle.OracleProblem(probs[0]).csr(with_detail=True)
        if graphs[0].E <= graphs[0].cap:
            parity.compare_full(graphs[0].to_numpy(), csr, probs[0].N, probs[0].nT, "f32")


def test_autotune_choice_keeps_results(tmp_path):
    probs = small_batch(seed=11, Q=4)
    pl = P.Planner.for_problem(probs[0], arith="f32", input="f32")
    dps = [P.to_device(p, input="f32") for p in probs]
    graphs = pl.build_batched(dps)
    ref = [g.to_numpy() for g in graphs]
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(pl, "test-small", reps=1, path=cache)
    assert res["tile"] in (32, 48, 64) and res["tchunks"] in (1, 2, 4, 8) and not res["cached"]
    graphs2 = pl.build_batched(dps)
    for r, g in zip(ref, graphs2):
        same_graph(g.to_numpy(), r)
    res2 = autotune.tune(pl, "test-small", reps=1, path=cache)
    assert res2["cached"] and res2["tile"] == res["tile"]
    for tile, ch, pipe in ((32, 1, 0), (44, 3, 0), (64, 8, 0), (64, 2, 1), (64, 5, 1), (64, 2, 2), (20, 4, 2)):
        pl.set_tile(tile, 0, ch, pipe)
        graphs3 = pl.build_batched(dps)
        for r, g in zip(ref, graphs3):
            same_graph(g.to_numpy(), r)


def test_batched_search_matches_oracle():
    probs = small_batch(seed=13, Q=6)
    pl = P.Planner.for_problem(probs[0], arith="f32", input="f32")
    dps = [P.to_device(p, input="f32") for p in probs]
    graphs = pl.build_batched(dps)
    res = pl.search_batched(dps, graphs)
    kinds = []
    for p, g, r in zip(probs, graphs, res):
        op = oracle.OracleProblem(p)
        csr = op.csr(with_detail=True)
        orc = oracle.search(op, csr, p.start_pos, p.goal_pos)
        # start/goal ids are not returned per query; the path's end points are
        if orc["path"] is None:
            assert r["status"] == P.PLAN_ERR_NO_PATH and r["path"] is None
            kinds.append("no-path")
            continue
        assert r["status"] == P.PLAN_OK
        kinds.append(parity.compare_search({"start": r["path"][0], "goal": r["path"][-1], "path": r["path"],
                                            "cost": r["cost"]}, orc, csr, "f32"))
    assert len(kinds) == 6


def test_one_query_replay_equals_build_edges():
    """One query prepared as a batch of one and its build replayed from a
    captured graph (the default benchmark step) gives plan_build_edges' graph
    bit for bit, also after its states and polytope bounds change in place."""
    prob = synth.triple_integrator_3d(seed=4, N=1500, K=12, nT=6)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pl = P.Planner.for_problem(prob, arith="f32", input="f32", stream=stream)
        dp = P.to_device(prob, input="f32")
        g = pl.build_edges(dp, cap=400 * prob.N)
        ref = g.to_numpy()
        pl.build_batched([dp], [g])
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            pl.build_batched_async()
        g.count.zero_()
        g.col.zero_()
        cg.replay()
        stream.synchronize()
        assert pl.wait() == P.PLAN_OK
        same_graph(g.to_numpy(), ref)
        # states moved and every bound loosened, in place
        rng = np.random.default_rng(5)
        prob.states = (prob.states + rng.normal(0.0, 0.05, prob.states.shape)).astype(prob.states.dtype)
        prob.b = (prob.b + 0.25).astype(prob.b.dtype)
        dp.states.copy_(torch.as_tensor(prob.states, dtype=torch.float32))
        dp.b.copy_(torch.as_tensor(prob.b, dtype=torch.float32))
        cg.replay()
        stream.synchronize()
        assert pl.wait() == P.PLAN_OK
        moved = g.to_numpy()
    fresh = P.Planner.for_problem(prob, arith="f32", input="f32")
    gf = fresh.build_edges(P.to_device(prob, input="f32"))
    same_graph(moved, gf.to_numpy())
    assert len(moved["col"]) != len(ref["col"])  # the replay did follow the new inputs
    csr = oracle.OracleProblem(prob).csr(with_detail=True)
    parity.compare_full(moved, csr, prob.N, prob.nT, "f32")
