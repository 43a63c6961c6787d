"""The replanning loop (Alg. 1 lines 3-4 every tick on the fixed graph of line
2): cut + search + path read-back replayed from one captured CUDA graph, with
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


def direct(pl, dp, g, obs, start, goal):
    out = pl.cut_edges(dp, g, P.obstacles_to_device(obs))
    buf = pl.alloc_search(dp.N)
    pl.search_async(dp, out, start, goal, buf)
    st = pl.wait()
    L = int(buf["path_len"].item())
    return {"status": st, "path": buf["path"][:L].cpu().tolist() if st == P.PLAN_OK else None,
            "cost": float(buf["cost"].item()), "edges": out.E, "csr": out.to_numpy()}


def test_replan_ticks_equal_direct_calls_and_oracle():
    prob, obs = synth.keepout_2d(3, N=600, n_obst=60)
    pl, dp, g, ctx = setup(prob)
    rp = P.Replanner(pl, dp, g, n_max=80, rows_max=8)
    rng = np.random.default_rng(3)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    for tick in range(6):
        cur = moved(obs, rng.normal(0.0, 0.05 * (tick + 1), size=(obs.n, 2)))
        start = prob.start_pos + rng.normal(0.0, 0.2, size=2)
        goal = prob.goal_pos + rng.normal(0.0, 0.2, size=2)
        r = rp.tick(cur, start, goal)
        d = direct(pl, dp, g, cur, start, goal)
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
    rp = P.Replanner(pl, dp, g, n_max=64, rows_max=8)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    for n in (40, 10, 0, 25):
        cur = subset(obs, n)
        r = rp.tick(cur, prob.start_pos, prob.goal_pos)
        d = direct(pl, dp, g, cur, prob.start_pos, prob.goal_pos)
        assert r["status"] == d["status"] and r["edges"] == d["edges"] and r["path"] == d["path"]
    assert r["info"]["cut_near"] < 5 * 40 * 500  # the padding slots are screened out by their boxes
    ctx.__exit__(None, None, None)


def test_replan_no_path_tick_then_recovery():
    prob, obs = synth.keepout_2d(5, N=500, n_obst=20)
    pl, dp, g, ctx = setup(prob)
    rp = P.Replanner(pl, dp, g, n_max=32, rows_max=8)
    rp.capture(obs, prob.start_pos, prob.goal_pos)
    wall = synth.Obstacles(np.array([0, 4], dtype=np.int32),
                           np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]),
                           np.array([100.0, 100.0, 100.0, 100.0]))   # covers everything: no edge left
    r = rp.tick(wall, prob.start_pos, prob.goal_pos)
    assert r["edges"] == 0 and (r["status"] == P.PLAN_ERR_NO_PATH or r["path"] == [r["info"]["start"]])
    r = rp.tick(obs, prob.start_pos, prob.goal_pos)
    d = direct(pl, dp, g, obs, prob.start_pos, prob.goal_pos)
    assert r["status"] == d["status"] and r["path"] == d["path"] and r["edges"] == d["edges"]
    ctx.__exit__(None, None, None)
