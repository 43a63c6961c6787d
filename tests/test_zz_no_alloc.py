"""The allocation-free search entry point, plan_search_noalloc.

Some callers cannot allocate device memory while they plan -- a replanning
loop with a hard per-tick deadline (cudaMalloc/cudaFree can block, cudaFree
synchronises the device), or a process whose device memory belongs to a pool
allocator.  For them the search keeps its scratch in a static device array of
the library.  These tests call it through the C ABI and check it against the
ordinary entry point, plan_search, on two calls in a row (different queries,
so a stale result from the shared scratch would show), with the parity bar
used elsewhere (exact start/goal and path, cost within 1e-12 relative for FP64
weights and 1e-5 for FP32); that a call after the first leaves the device's
free memory unchanged; and the largest accepted size, N = 65536, on a sparse
graph.  The file sorts last so a run that stops at the first failure has run
everything else.
"""
import numpy as np
import pytest

from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def _out(N):
    dev = torch.device("cuda")
    return {"path": torch.full((N,), -1, dtype=torch.int32, device=dev),
            "path_len": torch.zeros(1, dtype=torch.int32, device=dev),
            "cost": torch.zeros(1, dtype=torch.float64, device=dev),
            "status": torch.full((1,), -1, dtype=torch.int32, device=dev)}


@pytest.mark.parametrize("arith", ["f64", "f32"])
def test_noalloc_search_matches_plan_search_on_two_calls(arith):
    if arith == "f64":
        prob = synth.double_integrator_2d(1)
        queries = [(prob.start_pos, prob.goal_pos), (np.array([1.5, 8.5]), np.array([8.7, 1.2]))]
    else:
        prob = synth.triple_integrator_3d(2)
        queries = [(prob.start_pos, prob.goal_pos), (np.array([10.0, 4.0, 6.0]), np.array([3.0, 15.0, 12.0]))]
    pl = P.Planner.for_problem(prob, arith=arith, input=prob.dtype)
    dp = P.to_device(prob, input=prob.dtype)
    g = pl.build_edges(dp)
    tol = 1e-12 if arith == "f64" else 1e-5
    for s, gpos in queries:                       # two calls in a row
        ref = pl.search(dp, g, s, gpos)
        out = _out(dp.N)
        rc = P.search_noalloc(prob.model.m, prob.model.gamma, prob.dtype, arith == "f64", dp, g, s, gpos, out)
        assert rc == P.PLAN_OK
        torch.cuda.synchronize()
        st = int(out["status"].item())
        assert st == ref["status"]
        L = int(out["path_len"].item())
        if st == P.PLAN_OK:
            path = out["path"][:L].cpu().numpy().tolist()
            assert path == ref["path"]
            assert path[0] == ref["start"] and path[-1] == ref["goal"]
            c = float(out["cost"].item())
            assert abs(c - ref["cost"]) <= tol * max(1.0, abs(ref["cost"]))
        else:
            assert L == 0 and ref["path"] is None


def _check_against_plan_search(pl, dp, g, queries, m, gamma, input, w_f64, tol):
    for s, gpos in queries:                       # two calls in a row
        ref = pl.search(dp, g, s, gpos)
        out = _out(dp.N)
        rc = P.search_noalloc(m, gamma, input, w_f64, dp, g, s, gpos, out)
        assert rc == P.PLAN_OK
        torch.cuda.synchronize()
        st = int(out["status"].item())
        assert st == ref["status"]
        L = int(out["path_len"].item())
        if st == P.PLAN_OK:
            assert out["path"][:L].cpu().numpy().tolist() == ref["path"]
            c = float(out["cost"].item())
            assert abs(c - ref["cost"]) <= tol * max(1.0, abs(ref["cost"]))
        else:
            assert L == 0 and ref["path"] is None


def test_noalloc_search_allocates_nothing():
    prob = synth.double_integrator_2d(3)
    pl = P.Planner.for_problem(prob, arith="f64")
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    outs = [_out(dp.N) for _ in range(2)]
    m, gamma = prob.model.m, prob.model.gamma
    assert P.search_noalloc(m, gamma, "f64", True, dp, g, prob.start_pos, prob.goal_pos, outs[0]) == P.PLAN_OK
    torch.cuda.synchronize()                      # the first call has loaded the kernel and looked up the array
    free0, _ = torch.cuda.mem_get_info()
    assert P.search_noalloc(m, gamma, "f64", True, dp, g, prob.goal_pos, prob.start_pos, outs[1]) == P.PLAN_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(outs[0]["status"].item()) in (P.PLAN_OK, P.PLAN_ERR_NO_PATH)


def test_noalloc_search_at_its_largest_size():
    """N = 65536 (the static array's limit) on a sparse graph: ring edges plus two chords per vertex."""
    N = 65536
    rng = np.random.default_rng(5)
    states = np.zeros((N, 4))
    ang = 2 * np.pi * np.arange(N) / N
    states[:, 0], states[:, 1] = 100 * np.cos(ang), 100 * np.sin(ang)
    rows = []
    for i in range(N):
        rows.append(sorted({(i + 1) % N, (i + 97) % N, (i + 4099) % N}))
    col = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows])
    row_off = np.zeros(N + 1, dtype=np.int32)
    row_off[1:] = np.cumsum([len(r) for r in rows])
    w = rng.uniform(0.5, 2.0, size=col.shape[0])
    dev = torch.device("cuda")
    E = col.shape[0]
    g = P.Graph(N, torch.as_tensor(row_off).to(dev), torch.as_tensor(col).to(dev), torch.as_tensor(w).to(dev),
                torch.zeros(E, dtype=torch.uint8, device=dev), torch.ones(E, dtype=torch.int32, device=dev),
                torch.tensor([E], dtype=torch.int64, device=dev), E)
    st = torch.as_tensor(states).to(dev).contiguous()
    dp = P.DeviceProblem(N, 0, 1, st, None, None, None, np.array([1.0]), states[0, :2], states[N // 2, :2])
    pl = P.Planner(2, 2, 5, (2.0, 4.0), arith="f64", input="f64")
    queries = [(states[10, :2], states[40000, :2]), (states[65535, :2] * 1.01, states[123, :2])]
    _check_against_plan_search(pl, dp, g, queries, 2, 2, "f64", True, 1e-12)


def test_noalloc_search_rejects_more_vertices_than_its_scratch():
    prob = synth.double_integrator_2d(2, N=64, K=4)
    pl = P.Planner.for_problem(prob, arith="f64")
    dp = P.to_device(prob, input="f64")
    g = pl.build_edges(dp)
    big = P.DeviceProblem(65537, dp.K, dp.max_rows, dp.states, dp.poly_off, dp.A, dp.b, dp.T, dp.start_pos, dp.goal_pos)
    out = _out(16)
    rc = P.search_noalloc(2, 2, "f64", True, big, g, prob.start_pos, prob.goal_pos, out)
    assert rc == P.PLAN_ERR_CAPACITY
    assert int(out["status"].item()) == -1      # nothing was launched
