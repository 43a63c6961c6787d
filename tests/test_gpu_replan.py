"""The replanning loop (Algorithm 1's cutGraph and findPath every tick on the
graph its buildGraph made once): cut + search + path read-back replayed from one captured CUDA graph, with
moving obstacles and start/goal positions refreshed from pinned host memory.
Every tick must equal the direct (uncaptured) calls; two ticks are also
compared with the exact oracle."""
import numpy as np
import pytest

import oracle
import parity
from oracle import cut as OC
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu run happens on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def moved(obs, shift):
    """Every obstacle translated by shift[o] (b' = b + A d)."""
    A = np.asarray(obs.A).reshape(-1, 2)
    b = np.array(obs.b, dtype=np.float64)
    for o in range(obs.n):
        r0, r1 = obs.off[o], obs.off[o + 1]
        b[r0:r1] = b[r0:r1] + A[r0:r1] @ shift[o]
    return synth.Obstacles(np.asarray(obs.off), A.copy(), b)


def subset(obs, n):
    off = np.asarray(obs.off)[:n + 1]
    return synth.Obstacles(off, np.asarray(obs.A).reshape(-1, 2)[:off[-1]], np.asarray(obs.b)[:off[-1]])


def setup(prob):
    """A planner on its own stream (a captured graph cannot use the legacy
    default stream) and the fixed graph."""
    s = torch.cuda.Stream()
    ctx = torch.cuda.stream(s)
    ctx.__enter__()
    pl = P.Planner.for_problem(prob, stream=s)
    dp = P.to_device(prob)
    g = pl.build_edges(dp)
    return pl, dp, g, ctx


def direct(pl, dp, g, obs, start, goal, rooted="start"):
    """The same tick without capture: the cut, then a cold search (start-rooted
    plan_search, or goal-rooted plan_search_to without warm start)."""
    out = pl.cut_edges(dp, g, P.obstacles_to_device(obs))
    buf = pl.alloc_search(dp.N)
    if rooted == "start":
        pl.search_async(dp, out, start, goal, buf)
    else:
        ends = torch.as_tensor(np.concatenate([start, goal]), dtype=torch.float64).cuda()
        pl.search_to_async(dp, out, ends, buf, warm=False)
    st = pl.wait()
    L = int(buf["path_len"].item())
    return {"status": st, "path": buf["path"][:L].cpu().tolist() if st == P.PLAN_OK else None,
            "cost": float(buf["cost"].item()), "edges": out.E, "csr": out.to_numpy(), "info": pl.info()}


@pytest.mark.parametrize("warm", [True, False])
def test_replan_ticks_equal_direct_calls_and_oracle(warm):
    """Warm: the goal-rooted search warm-started from the previous tick must
    equal a cold goal-rooted search bit for bit (moving start, fixed goal, then
    a goal move that forces a cold start); cold: plan_search_at must equal
    plan_search."""
    prob, obs = synth.keepout_2d(3, N=600, n_obst=60)
    pl, dp, g, ctx = setup(prob)
    pl2 = P.Planner.for_problem(prob, stream=pl.stream)   # direct calls, own search state
    rp = P.Replanner(pl, dp, g, n_max=80, rows_max=8, warm=warm)
    rng = np.random.default_rng(3)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    goal = prob.goal_pos
    for tick in range(6):
        cur = moved(obs, rng.normal(0.0, 0.05 * (tick + 1), size=(obs.n, 2)))
        start = prob.start_pos + rng.normal(0.0, 0.2, size=2)
        if tick == 4:
            goal = prob.goal_pos + rng.normal(0.0, 0.5, size=2)
        r = rp.tick(cur, start, goal)
        d = direct(pl2, dp, g, cur, start, goal, rooted="goal" if warm else "start")
        assert r["status"] == d["status"] and r["edges"] == d["edges"]
        assert r["path"] == d["path"] and r["cost"] == d["cost"]
        if tick in (0, 5):
            orc = OC.cut(op, csr, cur.off, cur.A, cur.b)
            assert np.array_equal(d["csr"]["row_off"], orc["row_off"])
            parity.compare_rows(d["csr"], orc, range(prob.N), prob.nT, "f64")
            ocsr = {"row_off": orc["row_off"], "col": orc["col"], "w": orc["w"]}
            o = oracle.search(op, ocsr, start, goal)
            res = {"start": r["info"]["start"], "goal": r["info"]["goal"], "path": r["path"], "cost": r["cost"]}
            parity.compare_search(res, o, ocsr, "f64")
    ctx.__exit__(None, None, None)


def test_replan_with_fewer_obstacles_than_slots():
    prob, obs = synth.keepout_2d(4, N=500, n_obst=40)
    pl, dp, g, ctx = setup(prob)
    pl2 = P.Planner.for_problem(prob, stream=pl.stream)
    rp = P.Replanner(pl, dp, g, n_max=64, rows_max=8)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    for n in (40, 10, 0, 25):
        cur = subset(obs, n)
        r = rp.tick(cur, prob.start_pos, prob.goal_pos)
        d = direct(pl2, dp, g, cur, prob.start_pos, prob.goal_pos, rooted="goal")
        assert r["status"] == d["status"] and r["edges"] == d["edges"] and r["path"] == d["path"]
    assert r["info"]["cut_near"] < 5 * 40 * 500  # the padding slots are screened out by their boxes
    ctx.__exit__(None, None, None)


def test_replan_no_path_tick_then_recovery():
    prob, obs = synth.keepout_2d(5, N=500, n_obst=20)
    pl, dp, g, ctx = setup(prob)
    pl2 = P.Planner.for_problem(prob, stream=pl.stream)
    rp = P.Replanner(pl, dp, g, n_max=32, rows_max=8)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    wall = synth.Obstacles(np.array([0, 4], dtype=np.int32),
                           np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]),
                           np.array([100.0, 100.0, 100.0, 100.0]))   # covers everything: no edge left
    r = rp.tick(wall, prob.start_pos, prob.goal_pos)
    assert r["edges"] == 0 and (r["status"] == P.PLAN_ERR_NO_PATH or r["path"] == [r["info"]["start"]])
    r = rp.tick(obs, prob.start_pos, prob.goal_pos)
    d = direct(pl2, dp, g, obs, prob.start_pos, prob.goal_pos, rooted="goal")
    assert r["status"] == d["status"] and r["path"] == d["path"] and r["edges"] == d["edges"]
    ctx.__exit__(None, None, None)


def test_goal_rooted_search_matches_dijkstra_on_the_build_graph():
    """plan_search_to on a keep-in graph (2-D, FP64) against the oracle's
    Dijkstra: same start/goal, cost within 1e-12 relative, a shortest path."""
    prob = synth.double_integrator_2d(2)
    pl, dp, g, ctx = setup(prob)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    buf = pl.alloc_search(dp.N)
    ends = torch.as_tensor(np.concatenate([prob.start_pos, prob.goal_pos]), dtype=torch.float64).cuda()
    for warm in (False, True):
        pl.search_to_async(dp, g, ends, buf, warm=warm)
        st = pl.wait()
        info = pl.info()
        L = int(buf["path_len"].item())
        res = {"start": info["start"], "goal": info["goal"], "cost": float(buf["cost"].item()),
               "path": buf["path"][:L].cpu().tolist() if st == P.PLAN_OK else None}
        o = oracle.search(op, csr, prob.start_pos, prob.goal_pos)
        parity.compare_search(res, o, csr, "f64")
        if warm:
            assert info["search_iters"] == 1   # same graph, same goal: one confirming sweep
    ctx.__exit__(None, None, None)


def _search_to(pl, dp, out, start, goal, warm):
    buf = pl.alloc_search(dp.N)
    ends = torch.as_tensor(np.concatenate([start, goal]), dtype=torch.float64).cuda()
    pl.search_to_async(dp, out, ends, buf, warm=warm)
    st = pl.wait()
    L = int(buf["path_len"].item())
    return {"status": st, "path": buf["path"][:L].cpu().tolist() if st == P.PLAN_OK else None,
            "cost": float(buf["cost"].item()), "info": pl.info()}


@pytest.mark.parametrize("N,width", [(16000, 8.8), (30000, 12.0)])
def test_warm_start_after_a_stopped_call_on_the_cooperative_kernel(N, width):
    """Graphs above the on-chip (one cluster) size run the cooperative kernel:
    N = 16000 checks the chains in each block's shared memory, N = 30000 in
    global memory with one grid barrier per round.  A call stopped by the
    sweep limit leaves no warm state: the next warm call equals a cold one.
    Warm calls on moved obstacles equal cold calls bit for bit."""
    prob, obs = synth.keepout_2d(6, N=N, n_obst=300, width=width)
    pl, dp, g, ctx = setup(prob)
    pl2 = P.Planner.for_problem(prob, stream=pl.stream)
    rng = np.random.default_rng(6)
    start = prob.start_pos
    out = pl.cut_edges(dp, g, P.obstacles_to_device(obs))
    for v in rng.permutation(prob.N)[:100]:      # a goal the start reaches, 10 or more vertices away
        goal = prob.states[v, :2]
        first = _search_to(pl, dp, out, start, goal, warm=False)
        if first["status"] == P.PLAN_OK and len(first["path"]) >= 10:
            break
    assert first["status"] == P.PLAN_OK and len(first["path"]) >= 10
    pl.set_search_limits(max_sweeps=1)
    assert _search_to(pl, dp, out, start, goal, warm=False)["status"] == P.PLAN_ERR_TIMEOUT
    pl.set_search_limits(max_sweeps=0)
    again = _search_to(pl, dp, out, start, goal, warm=True)
    assert again["path"] == first["path"] and again["cost"] == first["cost"]
    assert again["info"]["search_iters"] > 1   # a warm start on the same graph would confirm in one sweep
    same = _search_to(pl, dp, out, start, goal, warm=True)
    assert same["path"] == first["path"] and same["info"]["search_iters"] == 1
    for tick in range(3):
        cur = moved(obs, rng.normal(0.0, 0.02, size=(obs.n, 2)))
        s = start + rng.normal(0.0, 0.3, size=2)
        out = pl.cut_edges(dp, g, P.obstacles_to_device(cur))
        r = _search_to(pl, dp, out, s, goal, warm=True)
        out2 = pl2.cut_edges(dp, g, P.obstacles_to_device(cur))
        c = _search_to(pl2, dp, out2, s, goal, warm=False)
        assert r["status"] == c["status"] and r["path"] == c["path"] and r["cost"] == c["cost"]
    ctx.__exit__(None, None, None)


def test_back_to_back_ticks_keep_one_in_flight():
    """Two tick_async calls without result() in between: the second waits for
    the first tick before it rewrites the staging buffers and drops the first
    tick's status, and the result equals a direct tick on the second
    obstacles."""
    prob, obs = synth.keepout_2d(5, N=500, n_obst=50)
    pl, dp, g, ctx = setup(prob)
    pl2 = P.Planner.for_problem(prob, stream=pl.stream)
    rp = P.Replanner(pl, dp, g, n_max=60, rows_max=8, warm=False)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    rng = np.random.default_rng(9)
    obs2 = moved(obs, rng.normal(0.0, 0.05, size=(obs.n, 2)))
    rp.tick(obs2, prob.start_pos, prob.goal_pos)      # sizes the cut's lists for both obstacle sets
    rp.tick(obs, prob.start_pos, prob.goal_pos)
    rp.tick_async(obs, prob.start_pos, prob.goal_pos)
    rp.tick_async(obs2, prob.start_pos, prob.goal_pos)
    r = rp.result()
    d = direct(pl2, dp, g, obs2, prob.start_pos, prob.goal_pos)
    assert r["status"] == d["status"] and r["path"] == d["path"] and r["edges"] == d["edges"]
    assert r["cost"] == d["cost"]
    ctx.__exit__(None, None, None)
