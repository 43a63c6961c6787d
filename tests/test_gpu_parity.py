"""GPU parity: the CUDA edge build and search (through the C ABI) against the
FP64 oracle on the same seeded inputs.  Bar: tests/parity.py."""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu run happens on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def gpu_build(prob, arith, input=None, planner=None, cap=None):
    input = input or prob.dtype
    pl = planner or P.Planner.for_problem(prob, arith=arith, input=input)
    dp = P.to_device(prob, input=input)
    g = pl.build_edges(dp, cap=cap)
    return pl, dp, g, pl.info()


def check_full(prob, arith, input=None, search=True):
    pl, dp, g, info = gpu_build(prob, arith, input)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    st = parity.compare_full(g.to_numpy(), csr, prob.N, prob.nT, arith)
    assert info["candidates"] == csr["candidates"]
    assert info["feasible"] == int(sum(bin(int(x)).count("1") for x in csr["mask"]))
    assert info["edges"] == len(csr["col"])
    res = None
    if search and prob.N > 0:
        r = pl.search(dp, g)
        orc = oracle.search(op, csr, prob.start_pos, prob.goal_pos)
        res = parity.compare_search(r, orc, csr, arith)
    return st, info, res


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_double_integrator_fp64_full(seed):
    """Plain method in FP64 (2-D double integrator, N=512, K=16, nT=8, p=5)."""
    st, info, res = check_full(synth.double_integrator_2d(seed), "f64")
    assert st["edges"] > 1000


@pytest.mark.parametrize("case", ["2d-1", "2d-4", "3d-f64", "2d-pos"])
def test_fp64_routes_agree_bit_for_bit(case):
    """The two FP64 routes -- FP32 pair kernels with FP64 re-check and an FP64
    cost pass (default), and the canonical FP64 pair kernel (pipeline 3) --
    give the same graph bit for bit (weights, durations, masks)."""
    if case.startswith("2d"):
        prob = synth.double_integrator_2d(int(case[-1]) if case[-1].isdigit() else 2)
    else:
        prob = synth.triple_integrator_3d(2, N=900, K=8, nT=12, dtype="f64")
    mdl = prob.model
    dp = P.to_device(prob, input="f64")
    graphs = []
    for pipe in (0, 3):
        pl = P.Planner(mdl.m, mdl.gamma, mdl.degree, mdl.bounds, arith="f64", input="f64",
                       cost_mode="pos" if case == "2d-pos" else "state")
        pl.set_tile(0, 0, 0, pipe)
        graphs.append(pl.build_edges(dp).to_numpy())
        info = pl.info()
        pl.close()
        if pipe == 3:
            assert info["rechecks"] == 0
    a, b = graphs
    for k in ("row_off", "col", "mask", "t"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["w"].view(np.uint64), b["w"].view(np.uint64))
    assert len(a["col"]) > 100


@pytest.mark.parametrize("seed", [1, 2])
def test_double_integrator_fp32_arith_on_fp64_inputs(seed):
    """FP32 margins + FP64 re-check on FP64 inputs must reproduce the FP64 bits."""
    st, info, res = check_full(synth.double_integrator_2d(seed), "f32", input="f64")
    assert st["edges"] > 1000


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_triple_integrator_fp32_small(seed):
    prob = synth.triple_integrator_3d(seed, N=700, K=6, nT=16)
    st, info, res = check_full(prob, "f32")
    assert st["edges"] > 100


def test_triple_integrator_fp32_full_size_all_rows():
    """Full-size 3-D workload (N=8192, K=64, nT=16, p=7, FP32), every row;
    seed 2 has an 18-vertex start-goal path."""
    prob = synth.triple_integrator_3d(2)
    pl, dp, g, info = gpu_build(prob, "f32")
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    st = parity.compare_full(g.to_numpy(), csr, prob.N, prob.nT, "f32")
    assert info["candidates"] == csr["candidates"]
    assert info["checks"] == csr["candidates"] * prob.nT
    r = pl.search(dp, g)
    orc = oracle.search(op, csr, prob.start_pos, prob.goal_pos)
    parity.compare_search(r, orc, csr, "f32")


@pytest.mark.parametrize("seed", [1, 3, 4, 5])
def test_triple_integrator_fp32_full_size_sampled_rows(seed):
    prob = synth.triple_integrator_3d(seed)
    pl, dp, g, info = gpu_build(prob, "f32")
    op = oracle.OracleProblem(prob)
    rows = np.unique(np.concatenate([np.arange(0, prob.N, 97), [0, prob.N - 1]])).astype(np.int32)
    e = op.edges(rows)
    parity.compare_rows(g.to_numpy(), e, rows, prob.nT, "f32")
    assert info["candidates"] == int(op.candidate_counts().sum())


@pytest.mark.parametrize("arith", ["f64", "f32"])
@pytest.mark.parametrize("degree", [3, 5])
def test_2d_degrees_and_single_big_polytope(arith, degree):
    """One polytope holding every state: many ragged tiles of one block."""
    prob = synth.double_integrator_2d(7, N=333, K=1, nT=5, degree=degree)
    check_full(prob, arith)


@pytest.mark.parametrize("arith", ["f64", "f32"])
def test_3d_degree5(arith):
    prob = synth.triple_integrator_3d(3, N=257, K=3, nT=7, degree=5, dtype="f64")
    check_full(prob, arith, input="f64")


@pytest.mark.parametrize("pipeline,tile", [(0, 64), (0, 8), (0, 28), (2, 64), (1, 64)])
def test_fp32_pair_kernels_loose_and_tight_bounds(pipeline, tile):
    """Every FP32 pair-kernel variant matches the oracle whether nearly every
    pair survives the reach screen (loose bounds: the survivor list overflows
    and threads take the extra pairs themselves), about a tenth does, or none."""
    for scale in (1000.0, 1.0, 0.05):
        prob = synth.triple_integrator_3d(7, N=600, K=5, nT=5)
        prob.model.bounds = tuple(float(b) * scale for b in prob.model.bounds)
        pl = P.Planner.for_problem(prob, arith="f32", input="f32")
        pl.set_tile(tile, 0, 0, pipeline)
        _, _, g, info = gpu_build(prob, "f32", planner=pl)
        csr = oracle.OracleProblem(prob).csr(with_detail=True)
        parity.compare_full(g.to_numpy(), csr, prob.N, prob.nT, "f32")
        assert info["edges"] == len(csr["col"])
        if scale == 1000.0:
            assert info["reach_pass"] > 0.9 * info["checks"]


def test_states_in_many_polytopes():
    """Rows of states that lie in more than 32 overlapping polytopes (the output
    pass merges such rows through the other segments' member lists) and in a
    handful of them (merged in shared memory)."""
    prob = synth.double_integrator_2d(9, N=260, K=40, nT=4)
    rng = np.random.default_rng(9)
    K = 40
    A = np.zeros((4 * K, 2))
    b = np.zeros(4 * K)
    for k in range(K):
        lo = rng.uniform(1.0, 4.0, 2)
        hi = rng.uniform(6.0, 9.0, 2)
        A[4 * k:4 * k + 4] = [[1, 0], [-1, 0], [0, 1], [0, -1]]
        b[4 * k:4 * k + 4] = [hi[0], -lo[0], hi[1], -lo[1]]
    prob.A, prob.b = A, b
    prob.poly_off = np.arange(0, 4 * K + 1, 4, dtype=np.int32)
    for i in range(prob.N):  # most states in the common core [4, 6]^2, some outside it
        prob.states[i, :2] = rng.uniform(4.0, 6.0, 2) if i % 3 else rng.uniform(1.5, 8.5, 2)
    prob.start_pos = np.array([4.5, 4.5])
    prob.goal_pos = np.array([5.5, 5.5])
    check_full(prob, "f64")
    check_full(prob, "f32", input="f64")


def test_maximum_polytope_count():
    """K = 1024 polytopes (the largest K a query takes): the item order ranks
    every polytope by tile area, with many ties and many polytopes without
    members or items; the graph equals the oracle's all the same."""
    prob = synth.double_integrator_2d(4, N=300, K=1024, nT=4)
    st, info, _ = check_full(prob, "f32", input="f64")
    assert info["edges"] > 0


@pytest.mark.parametrize("arith", ["f64", "f32"])
def test_minsnap_interior_points(arith):
    """Interior control points of minimal (gamma+1)-th-derivative energy
    (model flag interior = minsnap): the whole path against the oracle built
    on its own, independently derived minimum-energy tables."""
    prob = synth.double_integrator_2d(12, N=300, K=6)
    prob.model.interior = "minsnap"
    st, info, _ = check_full(prob, arith, input="f64")
    assert st["edges"] > 100
    prob3 = synth.triple_integrator_3d(12, N=500, K=5, nT=6)
    prob3.model.interior = "minsnap"
    st3, _, _ = check_full(prob3, arith, input="f32" if arith == "f32" else "f64")
    assert st3["edges"] > 50
    # a different curve: the edge set differs from the elevated reading's
    prob_e = synth.double_integrator_2d(12, N=300, K=6)
    e_csr = oracle.OracleProblem(prob_e).csr()
    m_csr = oracle.OracleProblem(prob).csr()
    assert not (np.array_equal(e_csr["row_off"], m_csr["row_off"]) and np.array_equal(e_csr["col"], m_csr["col"]))


@pytest.mark.parametrize("arith,input", [("f32", "f64"), ("f32", "f32")])
def test_near_duplicate_states_cost_accuracy(arith, input):
    """Pairs of nearly equal states: their FP32 cost halves cancel, so the
    FP32 cost is re-done in FP64 (cost conditioning test) and the weights
    still meet the 1e-5 bar."""
    prob = synth.double_integrator_2d(21, N=260, K=5)
    rng = np.random.default_rng(21)
    for i in range(0, 120, 2):  # state i+1 = state i moved by ~1e-3
        prob.states[i + 1] = prob.states[i] + rng.normal(0, 1e-3, prob.states.shape[1])
    if input == "f32":
        prob.states = prob.states.astype(np.float32).astype(np.float64)
    st, info, _ = check_full(prob, arith, input=input)
    assert st["max_rel_w"] <= 1e-5 and info["rechecks"] > 0


def test_nT_extremes():
    p1 = synth.double_integrator_2d(4, N=200, K=4, nT=1)
    check_full(p1, "f64")
    p32 = synth.double_integrator_2d(4, N=150, K=4, nT=32)
    check_full(p32, "f32", input="f64")


def test_tighten_and_position_cost():
    prob = synth.double_integrator_2d(5, N=300, K=6)
    prob.model.tighten = 0.05
    check_full(prob, "f64")
    prob2 = synth.triple_integrator_3d(5, N=400, K=4, nT=6)
    prob2.model.cost_mode = "pos"
    check_full(prob2, "f32")


def sixteen_row_problem():
    for seed in range(9, 200):
        prob = synth.make_problem("rows16", seed, synth.Model(2, 2, 5, (2.0, 4.0)), N=300, K=5,
                                  T=np.linspace(0.3, 2.0, 6), domain=(0.0, 8.0), side=(3.0, 6.0), max_cuts=12)
        if int(np.max(np.diff(prob.poly_off))) == 16:
            return prob
    raise AssertionError("no 16-row polytope drawn")


def test_sixteen_row_polytopes():
    prob = sixteen_row_problem()
    check_full(prob, "f64")
    check_full(prob, "f32", input="f64")


def test_degenerate_states():
    """Duplicate states, states outside every polytope, an empty polytope."""
    prob = synth.double_integrator_2d(6, N=240, K=5)
    prob.states[10] = prob.states[3]
    prob.states[11, :2] = [-50.0, -50.0]
    prob.states[12, :2] = [500.0, 500.0]
    # polytope 4 made empty: 0 <= -1
    lo, hi = prob.poly_off[4], prob.poly_off[5]
    prob.A[lo] = 0.0
    prob.b[lo] = -1.0
    check_full(prob, "f64")
    check_full(prob, "f32", input="f64")


def test_empty_and_tiny_inputs():
    for N, K in [(0, 3), (1, 3), (2, 1), (50, 0)]:
        prob = synth.double_integrator_2d(8, N=max(N, 1), K=max(K, 1), nT=3)
        prob.states = prob.states[:N]
        if K == 0:
            prob.poly_off = prob.poly_off[:1]
            prob.A = prob.A[:0]
            prob.b = prob.b[:0]
        pl = P.Planner.for_problem(prob, arith="f64")
        dp = P.to_device(prob, input="f64")
        g = pl.build_edges(dp)
        assert g.E == 0 or N >= 2
        csr = oracle.OracleProblem(prob).csr(with_detail=True)
        parity.compare_full(g.to_numpy(), csr, N, prob.nT, "f64")


def test_output_and_scratch_capacity_retry():
    """Too-small output and scratch: the device reports CAPACITY with the needed
    size, the binding grows and repeats, results still match."""
    prob = synth.double_integrator_2d(2)
    pl = P.Planner.for_problem(prob, arith="f64")
    dp = P.to_device(prob, input="f64")
    pl.build_edges(dp)                       # sizes the scratch
    g0 = pl.alloc_graph(prob.N, 1)
    pl.build_edges_async(dp, g0)
    assert pl.wait() == P.PLAN_ERR_CAPACITY and pl.last_info.detail == P.DET_OUTPUT
    need = pl.last_info.edges
    g = pl.build_edges(dp, graph=g0)
    assert g.E == need
    csr = oracle.OracleProblem(prob).csr(with_detail=True)
    parity.compare_full(g.to_numpy(), csr, prob.N, prob.nT, "f64")
    # scratch: every state in one polytope, many polytopes -> the first slot guess is too small
    big = synth.double_integrator_2d(3, N=600, K=64)
    lo, hi = big.poly_off[0], big.poly_off[1]
    big.A[lo:lo + 4] = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]], dtype=np.float64)
    big.b[lo:lo + 4] = [100.0, 100.0, 100.0, 100.0]
    big.A[lo + 4:hi] = [1.0, 0.0]
    big.b[lo + 4:hi] = 100.0
    pl2 = P.Planner.for_problem(big, arith="f32", input="f64")
    dp2 = P.to_device(big, input="f64")
    g2 = pl2.alloc_graph(big.N, 600 * 600)
    pl2.build_edges_async(dp2, g2)
    assert pl2.wait() == P.PLAN_ERR_CAPACITY and pl2.last_info.detail == P.DET_SLOTS
    g2 = pl2.build_edges(dp2, graph=g2)
    csr2 = oracle.OracleProblem(big).csr(with_detail=True)
    parity.compare_full(g2.to_numpy(), csr2, big.N, big.nT, "f32")


def test_host_argument_errors():
    prob = synth.double_integrator_2d(1, N=64, K=4)
    pl = P.Planner.for_problem(prob, arith="f64")
    dp = P.to_device(prob, input="f64")
    g = pl.alloc_graph(prob.N, 4096)
    import ctypes
    T = np.array([0.5])
    dpT = T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib = pl.lib
    ok = lambda rc: rc == P.PLAN_ERR_INVALID_ARG
    assert ok(lib.plan_build_edges(pl.ctx, -1, dp.states.data_ptr(), 1, dpT, dp.K, dp.poly_off.data_ptr(), dp.max_rows,
                                   dp.A.data_ptr(), dp.b.data_ptr(), ctypes.byref(g.cstruct())))
    assert ok(lib.plan_build_edges(pl.ctx, dp.N, dp.states.data_ptr(), 0, dpT, dp.K, dp.poly_off.data_ptr(), dp.max_rows,
                                   dp.A.data_ptr(), dp.b.data_ptr(), ctypes.byref(g.cstruct())))
    assert ok(lib.plan_build_edges(pl.ctx, dp.N, dp.states.data_ptr(), 1, dpT, dp.K, dp.poly_off.data_ptr(), 17,
                                   dp.A.data_ptr(), dp.b.data_ptr(), ctypes.byref(g.cstruct())))
    Tbad = np.array([-0.5])
    assert ok(lib.plan_build_edges(pl.ctx, dp.N, dp.states.data_ptr(), 1, Tbad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   dp.K, dp.poly_off.data_ptr(), dp.max_rows, dp.A.data_ptr(), dp.b.data_ptr(),
                                   ctypes.byref(g.cstruct())))
    assert ok(lib.plan_build_edges(pl.ctx, dp.N, None, 1, dpT, dp.K, dp.poly_off.data_ptr(), dp.max_rows,
                                   dp.A.data_ptr(), dp.b.data_ptr(), ctypes.byref(g.cstruct())))
    # a polytope with more rows than max_rows: device status UNSUPPORTED, no fault
    pl.build_edges_async(P.DeviceProblem(dp.N, dp.K, 2, dp.states, dp.poly_off, dp.A, dp.b, dp.T, dp.start_pos,
                                         dp.goal_pos), g)
    assert pl.wait() == P.PLAN_ERR_UNSUPPORTED
    # the context is still usable
    g2 = pl.build_edges(dp)
    assert g2.E > 0
    with pytest.raises(P.PlanError):
        P.Planner(4, 4, 7, [1, 1, 1, 1])


def test_search_no_path_and_timeout():
    """Disconnected start/goal -> NO_PATH on both sides; a sweep bound of 1 ->
    TIMEOUT reported by the device, and the context keeps working."""
    prob = synth.double_integrator_2d(3, N=200, K=2)
    # two far-apart boxes, no overlap
    prob.A[:] = 0
    for k, (cx, cy) in enumerate([(2.0, 2.0), (8.0, 8.0)]):
        lo = prob.poly_off[k]
        prob.A[lo:lo + 4] = [[1, 0], [-1, 0], [0, 1], [0, -1]]
        prob.b[lo:lo + 4] = [cx + 1, -(cx - 1), cy + 1, -(cy - 1)]
        prob.A[lo + 4:prob.poly_off[k + 1]] = [1, 0]
        prob.b[lo + 4:prob.poly_off[k + 1]] = cx + 1
    rng = np.random.default_rng(0)
    for i in range(prob.N):
        c = (2.0, 2.0) if i % 2 == 0 else (8.0, 8.0)
        prob.states[i, :2] = np.array(c) + rng.uniform(-0.9, 0.9, 2)
    prob.start_pos = np.array([2.0, 2.0])
    prob.goal_pos = np.array([8.0, 8.0])
    pl, dp, g, info = gpu_build(prob, "f64")
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    r = pl.search(dp, g)
    orc = oracle.search(op, csr, prob.start_pos, prob.goal_pos)
    assert parity.compare_search(r, orc, csr, "f64") == "no-path"
    assert r["status"] == P.PLAN_ERR_NO_PATH
    # sweep bound: 1 sweep cannot settle a multi-hop graph
    prob2 = synth.double_integrator_2d(1)
    pl2, dp2, g2, _ = gpu_build(prob2, "f64")
    pl2.set_search_limits(max_sweeps=1)
    out = pl2.alloc_search(prob2.N)
    pl2.search_async(dp2, g2, prob2.start_pos, prob2.goal_pos, out)
    assert pl2.wait() == P.PLAN_ERR_TIMEOUT
    pl2.set_search_limits(0, 0)
    r2 = pl2.search(dp2, g2)
    op2 = oracle.OracleProblem(prob2)
    csr2 = op2.csr(with_detail=True)
    parity.compare_search(r2, oracle.search(op2, csr2, prob2.start_pos, prob2.goal_pos), csr2, "f64")


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_search_random_queries(seed):
    """Several start/goal queries on one graph."""
    prob = synth.double_integrator_2d(seed)
    pl, dp, g, _ = gpu_build(prob, "f64")
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    rng = np.random.default_rng(seed)
    kinds = {}
    for _ in range(6):
        s, gpos = rng.uniform(0, 10, 2), rng.uniform(0, 10, 2)
        r = pl.search(dp, g, s, gpos)
        orc = oracle.search(op, csr, s, gpos)
        kind = parity.compare_search(r, orc, csr, "f64")
        kinds[kind] = kinds.get(kind, 0) + 1
    assert sum(kinds.values()) == 6
