"""Batching form at its stated size: the 256 uneven 3-D triple-integrator
queries of the benchmark (states log-uniform in 512-16384, 8-128 polytopes,
8-16 durations, degree 7, FP32) built in one replay of a captured CUDA graph
with the autotuned tiles, compared with the FP64 oracle; and one single-query
FP32 build at N = 16384.

What is compared (bar: tests/parity.py):
  * every query: start and goal vertices (the oracle's nearest vertex), and
    the rows of a sample (every row of a query with N <= 1024; rows 0, N-1
    and every 97th row otherwise) -- edge sets and masks bit-exact, weights
    within 1e-5, best duration where untied;
  * sixteen queries (the largest N, the largest K with 16 durations, the
    other 16-duration queries and a spread of smaller ones): the whole CSR
    and the batched search against the oracle's Dijkstra;
  * every other query's path: a walk over the GPU graph from the oracle's
    start vertex to its goal vertex whose FP64 weight sum is the reported
    cost (a property that holds at any size).
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import autotune  # noqa: E402
from paper_2411_13507_gb300 import plan as P  # noqa: E402

SEED = 2          # the benchmark's batch (bench.py --form batched)
Q = 256


def sample_rows(N: int) -> np.ndarray:
    if N <= 1024:
        return np.arange(N, dtype=np.int32)
    return np.unique(np.concatenate([np.arange(0, N, 97), [0, N - 1]])).astype(np.int32)


def full_set(probs) -> list:
    """Queries compared in full: largest N, largest-K 16-duration one, every 16-duration one, and a spread."""
    Ns = np.array([p.N for p in probs])
    pick = {int(np.argmax(Ns))}
    t16 = [q for q, p in enumerate(probs) if p.nT == 16]
    assert t16, "the batch must hold 16-duration queries"
    big = max(t16, key=lambda q: (probs[q].K >= 100, probs[q].N))
    pick.add(big)
    pick.update(t16)
    order = np.argsort(Ns)
    for q in order[:: max(1, len(order) // 12)]:
        if len(pick) >= 16:
            break
        pick.add(int(q))
    return sorted(pick)[:16]


@pytest.fixture(scope="module")
def batch():
    probs = synth.batched_queries(seed=SEED, Q=Q)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pl = P.Planner.for_problem(probs[0], arith="f32", input="f32", stream=stream)
        dps = [P.to_device(p, input="f32") for p in probs]
        graphs = pl.build_batched(dps)                      # sizes scratch and outputs
        tune = autotune.tune(pl, f"batched{Q}", reps=2)      # the benchmark's key and cache
        graphs = pl.build_batched(dps, graphs)               # prepared with the chosen tiles
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            pl.build_batched_async()
        for g in graphs:
            g.count.fill_(-1)
            g.row_off.fill_(-1)
        cg.replay()
        stream.synchronize()
        assert pl.wait() == P.PLAN_OK
        info = pl.info()
        res = pl.search_batched(dps, graphs)
    yield {"probs": probs, "graphs": [g.to_numpy() for g in graphs], "info": info, "tune": tune, "search": res}
    pl.close()


def test_batch_has_the_stated_shape(batch):
    probs = batch["probs"]
    Ns = [p.N for p in probs]
    assert len(probs) == Q and min(Ns) >= 512 and max(Ns) >= 12000
    assert max(p.K for p in probs) >= 100 and any(p.nT == 16 for p in probs)
    assert any(p.K >= 100 and p.nT == 16 and p.N >= 12000 for p in probs)
    assert batch["info"]["checks"] > 1e9


def test_every_query_sampled_rows_match_oracle(batch):
    stats = {"edges": 0, "tidx_checked": 0, "max_rel_w": 0.0, "rows": 0}
    for q, (p, g) in enumerate(zip(batch["probs"], batch["graphs"])):
        op = oracle.OracleProblem(p)
        rows = sample_rows(p.N)
        e = op.edges(rows, with_detail=True)
        s = parity.compare_rows(g, e, rows, p.nT, "f32")
        stats["edges"] += s["edges"]
        stats["tidx_checked"] += s["tidx_checked"]
        stats["max_rel_w"] = max(stats["max_rel_w"], s["max_rel_w"])
        stats["rows"] += len(rows)
        assert int(g["row_off"][-1]) == len(g["col"]), q
    print(f"\n256 queries, {stats['rows']} rows sampled: {stats['edges']} edges equal, "
          f"max weight rel err {stats['max_rel_w']:.2e}, tuned {batch['tune']}")
    assert stats["edges"] > 0


def test_sixteen_queries_full_csr_and_search(batch):
    kinds = []
    for q in full_set(batch["probs"]):
        p, g, r = batch["probs"][q], batch["graphs"][q], batch["search"][q]
        op = oracle.OracleProblem(p)
        csr = op.csr(with_detail=True)
        parity.compare_full(g, csr, p.N, p.nT, "f32")
        orc = oracle.search(op, csr, p.start_pos, p.goal_pos)
        if orc["path"] is None:
            assert r["status"] == P.PLAN_ERR_NO_PATH and r["path"] is None, q
            kinds.append("no-path")
            continue
        assert r["status"] == P.PLAN_OK, q
        kinds.append(parity.compare_search({"start": r["path"][0], "goal": r["path"][-1], "path": r["path"],
                                            "cost": r["cost"]}, orc, csr, "f32"))
    print(f"\nfull CSR + search on 16 queries: {kinds}")
    assert len(kinds) == 16


def test_every_query_path_is_a_walk_of_its_graph(batch):
    for q, (p, g, r) in enumerate(zip(batch["probs"], batch["graphs"], batch["search"])):
        op = oracle.OracleProblem(p)
        s, t = op.nearest(p.start_pos), op.nearest(p.goal_pos)
        if r["status"] == P.PLAN_ERR_NO_PATH:
            assert r["path"] is None
            continue
        assert r["status"] == P.PLAN_OK, (q, r["status"])
        path = r["path"]
        assert path[0] == s and path[-1] == t, q
        cost = 0.0
        for u, v in zip(path[:-1], path[1:]):
            a, b = int(g["row_off"][u]), int(g["row_off"][u + 1])
            k = np.searchsorted(g["col"][a:b], v)
            assert k < b - a and g["col"][a + k] == v, (q, u, v)
            cost = cost + float(g["w"][a + k])
        assert abs(cost - r["cost"]) <= 1e-12 * max(1.0, cost), (q, cost, r["cost"])


def test_single_query_n16384_fp32():
    p = synth.triple_integrator_3d(seed=3, N=16384)
    pl = P.Planner.for_problem(p, arith="f32", input="f32")
    dp = P.to_device(p, input="f32")
    g = pl.build_edges(dp).to_numpy()
    info = pl.info()
    op = oracle.OracleProblem(p)
    rows = sample_rows(p.N)
    s = parity.compare_rows(g, op.edges(rows, with_detail=True), rows, p.nT, "f32")
    assert s["edges"] > 0
    csr = op.csr(with_detail=False)
    assert info["candidates"] == csr["candidates"]
    assert np.array_equal(g["row_off"], csr["row_off"]) and np.array_equal(g["col"], csr["col"])
    assert np.array_equal(g["mask"], csr["mask"])
    rel = np.abs(g["w"] - csr["w"]) / csr["w"]
    assert rel.max() <= parity.TOL["f32"], rel.max()
    res = pl.search(dp, pl.build_edges(dp))
    orc = oracle.search(op, csr, p.start_pos, p.goal_pos)
    kind = parity.compare_search(res, orc, csr, "f32")
    print(f"\nN=16384: {info['checks']} checks, {len(csr['col'])} edges, sampled rows equal, search {kind}")
    pl.close()
