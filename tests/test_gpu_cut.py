"""GPU parity of the keep-out cut (Sec. III-B, Algorithm 2, Cut-QP) through the
C ABI against the exact oracle (oracle/cut.py) on the same seeded inputs.

Bar (tests/parity.py): the kept edge sets and masks bit-exact, weights within
1e-9 relative (FP64) or 1e-5 (FP32) of the oracle's FP64 costs, the duration
index wherever the oracle's best cost is untied.  A game that the FP64 pass
cannot certify either way (|delta*| at the FP64 rounding level) is a declared
tie; these inputs must produce none."""
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


def build(prob, arith, input=None):
    input = input or prob.dtype
    pl = P.Planner.for_problem(prob, arith=arith, input=input)
    dp = P.to_device(prob, input=input)
    g = pl.build_edges(dp)
    return pl, dp, g


def run_cut(prob, obs, arith, input=None):
    input = input or prob.dtype
    pl, dp, g = build(prob, arith, input)
    E_in = g.E
    out = pl.cut_edges(dp, g, P.obstacles_to_device(obs, input=input))
    return pl, dp, g, out, pl.info(), E_in


def check(prob, obs, arith, input=None, rows=None):
    pl, dp, g, out, info, E_in = run_cut(prob, obs, arith, input)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    orc = OC.cut(op, csr, obs.off, obs.A, obs.b, rows=rows)
    gpu = out.to_numpy()
    if rows is None:
        assert np.array_equal(gpu["row_off"], orc["row_off"]), "row offsets differ"
        rows = range(prob.N)
    st = parity.compare_rows(gpu, orc, rows, prob.nT, arith)
    assert info["cut_ties"] == 0
    assert info["cut_units"] == int(sum(bin(int(x)).count("1") for x in csr["mask"]))
    assert info["cut_box"] + info["cut_near"] == info["cut_tests"]
    assert info["cut_step1"] + info["cut_step2"] + info["cut_games"] <= info["cut_near"]
    return st, info, orc, gpu, g, out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_keepout_fp64_all_rows(seed):
    """2-D double integrator, N=600, 60 obstacles, FP64: every row."""
    prob, obs = synth.keepout_2d(seed, N=600, n_obst=60)
    st, info, orc, gpu, g, out = check(prob, obs, "f64")
    assert 0 < len(gpu["col"]) < g.E
    assert orc["steps"][3] > 0 and info["cut_games"] > 0


@pytest.mark.parametrize("seed", [1, 2])
def test_keepout_fp32_all_rows(seed):
    prob, obs = synth.keepout_2d(seed, N=600, n_obst=60, dtype="f32")
    st, info, orc, gpu, g, out = check(prob, obs, "f32")
    assert 0 < len(gpu["col"]) < g.E


def test_keepout_full_size_sampled_rows():
    """The full keep-out workload (N=5000, 500 obstacles, about 46,000 edges),
    every 50th row against the oracle."""
    prob, obs = synth.keepout_2d(1)
    st, info, orc, gpu, g, out = check(prob, obs, "f64", rows=np.arange(0, prob.N, 50))
    assert st["edges"] > 200 and info["cut_tests"] > 10_000_000


def test_several_durations_recost_when_best_is_cut():
    """nT=8 keep-in graph plus obstacles: edges whose cheapest duration is cut
    get the cheapest remaining one, re-costed in FP64."""
    prob = synth.double_integrator_2d(3)
    obs = synth.obstacles(3, 40, 2, (0.0, 10.0), (0.2, 0.8), 3)
    st, info, orc, gpu, g, out = check(prob, obs, "f64")
    gin = g.to_numpy()
    src_in = np.repeat(np.arange(prob.N), np.diff(gin["row_off"]))
    src_out = np.repeat(np.arange(prob.N), np.diff(gpu["row_off"]))
    key_in = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(src_in, gin["col"]))}
    moved = sum(int(gin["t"][key_in[(int(i), int(j))]] != t) for i, j, t in zip(src_out, gpu["col"], gpu["t"]))
    assert moved > 0 and st["tidx_checked"] > 0


@pytest.mark.parametrize("seed", [1, 4])
def test_triple_integrator_fp32_cut(seed):
    """3-D triple integrator (p=7, nT=6, FP32) against 3-D obstacles."""
    prob = synth.triple_integrator_3d(seed, N=300, K=6, nT=6)
    # boxes near random states (the free polytopes fill a small part of the domain)
    rng = np.random.default_rng(seed)
    ctr = prob.states[rng.choice(prob.N, 40, replace=False), :3] + rng.uniform(-1.0, 1.0, size=(40, 3))
    half = rng.uniform(0.2, 0.6, size=(40, 3))
    eye = np.concatenate([np.eye(3), -np.eye(3)])
    A = np.tile(eye, (40, 1))
    b = np.concatenate([np.concatenate([c + h, -(c - h)]) for c, h in zip(ctr, half)])
    obs = synth.Obstacles(np.arange(0, 6 * 40 + 1, 6, dtype=np.int32), A.astype(np.float32).astype(np.float64),
                          b.astype(np.float32).astype(np.float64))
    st, info, orc, gpu, g, out = check(prob, obs, "f32")
    bits = lambda m: int(sum(bin(int(x)).count("1") for x in m))
    assert 0 < bits(gpu["mask"]) < bits(g.to_numpy()["mask"])


def regular_polygons(n, rows, centers, radius):
    th = 2 * np.pi * (np.arange(rows) + 0.25) / rows
    nrm = np.stack([np.cos(th), np.sin(th)], axis=1)
    A = np.tile(nrm, (n, 1))
    b = np.concatenate([nrm @ c + radius for c in centers])
    return synth.Obstacles(np.arange(0, rows * n + 1, rows, dtype=np.int32), A, b)


def test_sixteen_row_obstacles():
    prob, _ = synth.keepout_2d(4, N=500, n_obst=1)
    rng = np.random.default_rng(4)
    obs = regular_polygons(30, 16, rng.uniform(0.0, 5.0, size=(30, 2)), 0.08)
    check(prob, obs, "f64")


def test_no_obstacles_copies_the_graph():
    prob, _ = synth.keepout_2d(5, N=400, n_obst=1)
    obs = synth.Obstacles(np.zeros(1, dtype=np.int32), np.zeros((0, 2)), np.zeros(0))
    pl, dp, g, out, info, E_in = run_cut(prob, obs, "f64")
    a, b = g.to_numpy(), out.to_numpy()
    for k in ("row_off", "col", "w", "t", "mask"):
        assert np.array_equal(a[k], b[k]), k
    assert info["cut_tests"] == 0


def test_whole_space_and_covering_obstacles_cut_everything():
    prob, _ = synth.keepout_2d(6, N=400, n_obst=1)
    empty = synth.Obstacles(np.array([0, 0], dtype=np.int32), np.zeros((0, 2)), np.zeros(0))
    big = synth.Obstacles(np.array([0, 4], dtype=np.int32),
                          np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]), np.array([100.0, 100.0, 100.0, 100.0]))
    for obs in (empty, big):
        pl, dp, g, out, info, E_in = run_cut(prob, obs, "f64")
        assert E_in > 0 and out.E == 0
        assert int(out.row_off.abs().sum().item()) == 0


def test_empty_graph():
    prob, obs = synth.keepout_2d(7, N=1, n_obst=5)
    pl, dp, g, out, info, E_in = run_cut(prob, obs, "f64")
    assert E_in == 0 and out.E == 0 and info["cut_units"] == 0


def test_output_capacity_reports_the_count():
    prob, obs = synth.keepout_2d(8, N=600, n_obst=60)
    pl, dp, g = build(prob, "f64")
    do = P.obstacles_to_device(obs)
    full = pl.cut_edges(dp, g, do)
    small = pl.alloc_graph(prob.N, max(1, full.E // 2))
    pl.cut_edges_async(dp, g, do, small)
    assert pl.wait() == P.PLAN_ERR_CAPACITY
    assert small.E == full.E


def test_obstacle_with_too_many_rows_is_unsupported():
    prob, _ = synth.keepout_2d(9, N=300, n_obst=1)
    obs = regular_polygons(2, 8, np.array([[1.0, 1.0], [2.0, 2.0]]), 0.1)
    pl, dp, g = build(prob, "f64")
    do = P.obstacles_to_device(obs)
    do.max_rows = 4  # declared bound below the real row count
    out = pl.alloc_graph(prob.N, g.cap)
    pl.cut_edges_async(dp, g, do, out)
    assert pl.wait() == P.PLAN_ERR_UNSUPPORTED


def test_cut_then_search_matches_oracle():
    """findPath on the cut graph (Algorithm 1's cutGraph, then findPath)."""
    prob, obs = synth.keepout_2d(2, N=600, n_obst=60)
    pl, dp, g, out, info, E_in = run_cut(prob, obs, "f64")
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    orc = OC.cut(op, csr, obs.off, obs.A, obs.b)
    ocsr = {"row_off": orc["row_off"], "col": orc["col"], "w": orc["w"]}
    r = pl.search(dp, out)
    o = oracle.search(op, ocsr, prob.start_pos, prob.goal_pos)
    parity.compare_search(r, o, ocsr, "f64")


def test_near_tie_games_go_through_the_fp64_pass():
    """Curves that miss or graze an obstacle corner by 1e-7 (far inside the
    FP32 bands): the FP32 passes cannot decide them, the canonical FP64 pass
    must, and no game may end as a tie."""
    prob, _ = synth.keepout_2d(11, N=60, n_obst=1, width=4.0)
    prob.states[:, 2:] = 0.0                 # at rest: every curve is a segment
    prob.model.bounds = (50.0, 500.0)        # every pair reachable
    rng = np.random.default_rng(11)
    A, b, off = [], [], [0]
    for k in range(24):
        i, j = rng.choice(prob.N, 2, replace=False)
        p, q = prob.states[i, :2], prob.states[j, :2]
        dvec = q - p
        nrm = np.array([dvec[1], -dvec[0]]) / np.hypot(*dvec)
        d = 1e-7 if k % 2 == 0 else -1e-7   # miss / overlap by 1e-7
        c = 0.5 * (p + q) + d * nrm
        sx, sy = np.sign(nrm[0]) or 1.0, np.sign(nrm[1]) or 1.0
        # the quadrant at corner c facing away from the segment
        A += [[sx, 0.0], [-sx, 0.0], [0.0, sy], [0.0, -sy]]
        b += [sx * c[0] + 0.3, -sx * c[0], sy * c[1] + 0.3, -sy * c[1]]
        off.append(off[-1] + 4)
    obs = synth.Obstacles(np.array(off, dtype=np.int32), np.array(A), np.array(b))
    st, info, orc, gpu, g, out = check(prob, obs, "f64")
    assert info["cut_lp64"] > 0 and info["cut_ties"] == 0
