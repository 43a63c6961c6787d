"""GPU parity of the MPC refinement QP (plan_mpc_qp) and of the nearest
obstacle's plane (plan_nearest_planes) against the FP64 oracles
(oracle/mpc.py, oracle/planes.py).

Bar.  Both sides compute the unique optimum of the same strictly convex QP
in FP64 by different exact methods (GPU: condensed inputs, dual active set;
oracle: node states and inputs with the dynamics as equalities, primal
active set), so they differ by rounding amplified by the conditioning of
the KKT system: the tests allow 1e-7 (1 + |x|) on the nodes, 1e-6 (1 + |u|)
on the inputs (the inputs of a chain of integrators are the g-th
differences of the nodes divided by dt^g, so their error is larger by about
dt^-g), require the GPU's objective to be its own (x, u) evaluated (1e-10
relative) and the two optimal values to agree to 1e-6 relative (first order
in the solution's error), and require the same status.
The planes passed to both sides are the same float32 values."""
import numpy as np
import pytest

from mpc_cases import instance, objective, solve, with_keepin
from oracle import mpc as OM
from oracle import planes as OP
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu run happens on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def planner(m, g, p, bounds):
    return P.Planner(m, g, p, tuple(bounds[:g]), arith="f64", input="f64")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def run_batch(insts):
    """One plan_mpc_qp launch over every instance (same model, dt, weights,
    keep-in rows)."""
    i0 = insts[0]
    m, g, p, H = i0["m"], i0["g"], i0["p"], i0["ref"].shape[0] - 1
    pl = planner(m, g, p, i0["bounds"])
    prm = pl.mpc_params(H, i0["dt"], i0["Q"], i0["F"], i0["R"], i0["V"], i0.get("keepin_A"), i0.get("keepin_b"))
    B = len(insts)
    dev = torch.device("cuda")
    x0 = torch.tensor(np.stack([t["x0"] for t in insts]), dtype=torch.float64, device=dev)
    ref = torch.tensor(np.stack([t["ref"] for t in insts]), dtype=torch.float64, device=dev)
    planes = torch.tensor(np.stack([t["planes"] for t in insts]), dtype=torch.float32, device=dev)
    out = pl.alloc_mpc(B, H)
    pl.mpc_qp_async(prm, x0, ref, planes, out)
    assert pl.wait() == P.PLAN_OK
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(gpu, b, inst):
    inst = dict(inst, planes=f32(inst["planes"]))
    orc = solve(inst)
    st = int(gpu["status"][b])
    if orc["status"] == OM.INFEASIBLE:
        assert st == P.PLAN_MPC_INFEASIBLE
        return None
    assert orc["status"] == OM.OK and st == P.PLAN_MPC_OK, (orc["status"], st)
    x, u = gpu["x"][b], gpu["u"][b]
    assert np.abs(x - orc["x"]).max() <= 1e-7 * (1 + np.abs(orc["x"]).max()), np.abs(x - orc["x"]).max()
    assert np.abs(u - orc["u"]).max() <= 1e-6 * (1 + np.abs(orc["u"]).max()), np.abs(u - orc["u"]).max()
    # the GPU's objective is its own (x, u) evaluated exactly; the optimal
    # values agree to first order in the solution's error (the gradient at a
    # constrained optimum is not zero)
    assert abs(gpu["obj"][b] - objective(inst, x, u)) <= 1e-10 * (1 + abs(orc["obj"]))
    assert abs(gpu["obj"][b] - orc["obj"]) <= 1e-6 * (1 + abs(orc["obj"]))
    return orc


def cut_in(inst, seed, depth=0.015):
    """Planes of two segments moved into the reference, so that rows bind."""
    inst = dict(inst, planes=inst["planes"].copy())
    m, H = inst["m"], inst["ref"].shape[0] - 1
    rng = np.random.default_rng(seed)
    for k in rng.choice(np.arange(1, H), size=2, replace=False):
        inst["planes"][k, m] += depth
    return inst


@pytest.mark.parametrize("m,g,p,keepin", [(2, 2, 5, False), (2, 2, 5, True), (3, 3, 7, False), (3, 3, 7, True)])
def test_batch_against_oracle(m, g, p, keepin):
    insts = []
    for s in range(12):
        t = instance(100 * m + s, m=m, g=g, p=p, H=8)
        if s % 3 == 1:
            t = cut_in(t, s)
        if s % 3 == 2:
            t = dict(t, planes=np.zeros_like(t["planes"]))   # no safety rows at all
        insts.append(t)
    if keepin:
        # one keep-in box for the whole batch: the union of the references' extents
        boxes = [with_keepin(t, 0.01) for t in insts]
        KA = boxes[0]["keepin_A"]
        Kb = np.max(np.stack([bx["keepin_b"] for bx in boxes]), axis=0)
        insts = [dict(t, keepin_A=KA, keepin_b=Kb) for t in insts]
    gpu = run_batch(insts)
    active = 0
    for b, t in enumerate(insts):
        orc = compare(gpu, b, t)
        if orc is not None:
            active += len(orc["active"])
    assert active > 0   # some rows bind in the batch


def test_largest_horizon_and_single_problem():
    """m H = 64 inputs (the limit), B = 1."""
    t = cut_in(instance(7, H=32, dt=0.05), 7)
    gpu = run_batch([t])
    compare(gpu, 0, t)


def test_infeasible_and_feasible_in_one_batch():
    good = instance(11)
    bad = instance(12)
    bad["planes"][3, :2] = [1.0, 0.0]
    bad["planes"][3, 2] = 1e3
    gpu = run_batch([good, bad, good])
    compare(gpu, 0, good)
    assert int(gpu["status"][1]) == P.PLAN_MPC_INFEASIBLE
    compare(gpu, 2, good)


def test_host_errors_and_empty_batch():
    t = instance(13)
    pl = planner(2, 2, 5, t["bounds"])
    out = pl.alloc_mpc(0, 8)
    prm = pl.mpc_params(8, 0.1, t["Q"], t["F"], t["R"], t["V"])
    e = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    pl.mpc_qp_async(prm, e, torch.empty((0, 9, 4), dtype=torch.float64, device="cuda"),
                    torch.empty((0, 8, 3), dtype=torch.float32, device="cuda"), out)
    assert pl.wait() == P.PLAN_OK
    for bad in (pl.mpc_params(1, 0.1, t["Q"], t["F"], t["R"], t["V"]),          # H < gamma
                pl.mpc_params(33, 0.1, t["Q"], t["F"], t["R"], t["V"]),         # m H > 64
                pl.mpc_params(8, -1.0, t["Q"], t["F"], t["R"], t["V"]),         # dt <= 0
                pl.mpc_params(8, 0.1, np.zeros(4), t["F"], t["R"], t["V"])):    # weight 0
        with pytest.raises(RuntimeError):
            pl.mpc_qp_async(bad, e, e, e, out)


def nodes_and_obstacles(seed, B, H):
    """References of the keep-out workload's scale and obstacles near them."""
    prob, obs = synth.keepout_2d(seed, N=400, n_obst=60, width=5.0)
    insts = [instance(1000 * seed + b, H=H) for b in range(B)]
    return insts, obs


def test_nearest_planes_against_oracle():
    insts, obs = nodes_and_obstacles(3, 6, 8)
    pts = np.concatenate([t["ref"][:8, :2] for t in insts])
    pl = planner(2, 2, 5, insts[0]["bounds"])
    dev = torch.device("cuda")
    do = P.obstacles_to_device(obs, input="f64")
    plane = torch.empty((pts.shape[0], 3), dtype=torch.float32, device=dev)
    near = torch.empty(pts.shape[0], dtype=torch.int32, device=dev)
    pl.nearest_planes_async(torch.tensor(pts, dtype=torch.float64, device=dev), do, plane, near)
    assert pl.wait() == P.PLAN_OK
    plane, near = plane.cpu().numpy(), near.cpu().numpy()
    orc = OP.planes(pts, obs.off, obs.A, obs.b)
    for i in range(pts.shape[0]):
        d = np.sort(orc["dist"][i])
        if near[i] != orc["nearest"][i]:
            assert d[1] - d[0] <= 1e-4
            continue
        o = orc["nearest"][i]
        if orc["dist"][i, o] > 1e-3:
            assert np.abs(plane[i, :2] - orc["plane"][i, o, :2]).max() <= 1e-4
            assert abs(plane[i, 2] - orc["plane"][i, o, 2]) <= 1e-4 * (1 + np.abs(pts).max())
        # the node lies on the positive side of its plane
        assert plane[i, :2].astype(np.float64) @ pts[i] - plane[i, 2] >= -1e-5


def test_sqp_rounds_against_oracle():
    """Three SQP rounds (planes at the current nodes, then the QP): every
    round's QP equals the oracle's on the same planes, and the loop driven by
    mpc_refine_async ends at the same nodes."""
    insts, obs = nodes_and_obstacles(4, 8, 8)
    i0 = insts[0]
    H = 8
    pl = planner(2, 2, 5, i0["bounds"])
    dev = torch.device("cuda")
    do = P.obstacles_to_device(obs, input="f64")
    prm = pl.mpc_params(H, i0["dt"], i0["Q"], i0["F"], i0["R"], i0["V"])
    x0 = torch.tensor(np.stack([t["x0"] for t in insts]), dtype=torch.float64, device=dev)
    ref = torch.tensor(np.stack([t["ref"] for t in insts]), dtype=torch.float64, device=dev)
    B = len(insts)
    out = pl.alloc_mpc(B, H)
    planes = torch.empty((B, H, 3), dtype=torch.float32, device=dev)
    cur = ref
    for rnd in range(3):
        nodes = cur[:, :H, :2].contiguous().view(B * H, 2)
        pl.nearest_planes_async(nodes, do, planes.view(B * H, 3))
        pl.mpc_qp_async(prm, x0, ref, planes, out)
        assert pl.wait() == P.PLAN_OK
        g = {k: v.cpu().numpy() for k, v in out.items()}
        assert np.array_equal(g["nodes"], g["x"][:, :H, :2])   # the next round's points
        pn = planes.cpu().numpy().astype(np.float64)
        for b, t in enumerate(insts):
            compare(g, b, dict(t, planes=pn[b]))
        cur = out["x"].clone()
    last = g["x"].copy()
    out2 = pl.alloc_mpc(B, H)
    pl.mpc_refine_async(prm, x0, ref, do, out2, sqp_iters=3)
    assert pl.wait() == P.PLAN_OK
    assert np.array_equal(out2["x"].cpu().numpy(), last)


def test_factor_cache_follows_the_weights():
    """One context, three calls: weights W1, W2 (the Hessian's factor must be
    recomputed), W1 again -- each against the oracle."""
    insts = [cut_in(instance(40 + s), s) for s in range(4)]
    i0 = insts[0]
    H = i0["ref"].shape[0] - 1
    pl = planner(2, 2, 5, i0["bounds"])
    dev = torch.device("cuda")
    x0 = torch.tensor(np.stack([t["x0"] for t in insts]), dtype=torch.float64, device=dev)
    ref = torch.tensor(np.stack([t["ref"] for t in insts]), dtype=torch.float64, device=dev)
    planes = torch.tensor(np.stack([t["planes"] for t in insts]), dtype=torch.float32, device=dev)
    for Q in (i0["Q"], 3.0 * i0["Q"], i0["Q"]):
        prm = pl.mpc_params(H, i0["dt"], Q, i0["F"], i0["R"], i0["V"])
        out = pl.alloc_mpc(len(insts), H)
        pl.mpc_qp_async(prm, x0, ref, planes, out)
        assert pl.wait() == P.PLAN_OK
        g = {k: v.cpu().numpy() for k, v in out.items()}
        for b, t in enumerate(insts):
            compare(g, b, dict(t, Q=Q))
