"""Pins for the MPC refinement oracle (oracle/mpc.py).  Expected values come
from the kinematics of a constant input (the discretisation), brute-force
enumeration of active sets on tiny QPs, clipping (separable box QPs), an
unconstrained least-squares solution written in the condensed variables
(independent of the oracle's uncondensed active-set route), the objective
recomputed term by term, dense sampling of every segment's Bezier curve and
derivatives against the constraints, the KKT conditions by non-negative
least squares, and planted mistakes."""
from itertools import combinations

import numpy as np
import pytest

from mpc_cases import bezier_points, instance, kin_step, objective, segment_control_points, solve, with_keepin
from oracle import mpc


@pytest.mark.parametrize("m,g", [(2, 2), (3, 3), (1, 4)])
def test_discretisation_is_the_constant_input_kinematics(m, g):
    rng = np.random.default_rng(m * 10 + g)
    A, B = mpc.discretize(m, g, 0.37)
    for _ in range(20):
        x = rng.normal(size=m * g)
        u = rng.normal(size=m)
        assert np.allclose(A @ x + B @ u, kin_step(x, u, m, g, 0.37), rtol=1e-13, atol=1e-13)


def brute_force_qp(P, q, Aeq, beq, Ain, bin_):
    """The optimum of a strictly convex QP as the KKT point among all active
    sets (feasible, non-negative multipliers)."""
    nz, ne, ni = P.shape[0], Aeq.shape[0], Ain.shape[0]
    best = None
    for k in range(0, min(ni, nz - ne) + 1):
        for S in combinations(range(ni), k):
            AW = np.concatenate([Aeq, Ain[list(S)]])
            bW = np.concatenate([beq, bin_[list(S)]])
            K = np.block([[P, AW.T], [AW, np.zeros((AW.shape[0], AW.shape[0]))]])
            if abs(np.linalg.det(K)) < 1e-12:
                continue
            sol = np.linalg.solve(K, np.concatenate([-q, bW]))
            z, lam = sol[:nz], sol[nz:]
            if np.all(Ain @ z - bin_ <= 1e-9) and np.all(lam[ne:] >= -1e-9):
                if best is not None:
                    assert np.allclose(best, z, atol=1e-8)   # unique optimum
                best = z
    return best


@pytest.mark.parametrize("seed", range(12))
def test_qp_solver_against_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    nz = 4
    M = rng.normal(size=(nz, nz))
    P = M @ M.T + 0.5 * np.eye(nz)
    q = rng.normal(size=nz) * 3
    Aeq = rng.normal(size=(1, nz))
    beq = rng.normal(size=1)
    Ain = rng.normal(size=(7, nz))
    bin_ = rng.uniform(0.1, 1.0, size=7)
    # a feasible point for the equality row too: shift beq so that z = 0 is feasible
    beq = np.zeros(1)
    st, z, W, y, mu = mpc.solve_qp(P, q, Aeq, beq, Ain, bin_)
    assert st == mpc.OK
    zb = brute_force_qp(P, q, Aeq, beq, Ain, bin_)
    assert np.allclose(z, zb, atol=1e-9)


def test_box_qp_is_clipping():
    rng = np.random.default_rng(7)
    for _ in range(20):
        nz = 6
        c = rng.normal(size=nz) * 2
        lo, hi = -rng.uniform(0.1, 1, size=nz), rng.uniform(0.1, 1, size=nz)
        P = 2 * np.eye(nz)
        q = -2 * c
        Ain = np.concatenate([np.eye(nz), -np.eye(nz)])
        bin_ = np.concatenate([hi, -lo])
        st, z, W, y, mu = mpc.solve_qp(P, q, np.zeros((0, nz)), np.zeros(0), Ain, bin_)
        assert st == mpc.OK and np.allclose(z, np.clip(c, lo, hi), atol=1e-12)


def test_infeasible_qp():
    P = np.eye(2)
    Ain = np.array([[1.0, 0.0], [-1.0, 0.0]])
    bin_ = np.array([-1.0, -1.0])       # x <= -1 and x >= 1
    st, *_ = mpc.solve_qp(P, np.zeros(2), np.zeros((0, 2)), np.zeros(0), Ain, bin_)
    assert st == mpc.INFEASIBLE


# ---------------------------------------------------------------------------
# MPC instances


@pytest.mark.parametrize("seed,m,g,p,keepin", [(1, 2, 2, 5, False), (2, 2, 2, 5, False), (3, 2, 2, 5, True),
                                               (4, 3, 3, 7, False), (5, 3, 3, 7, True)])
def test_mpc_solution_properties(seed, m, g, p, keepin):
    inst = instance(seed, m=m, g=g, p=p)
    if keepin:
        inst = with_keepin(inst)
    r = solve(inst)
    assert r["status"] == mpc.OK
    x, u = r["x"], r["u"]
    m, g, p, dt, H = inst["m"], inst["g"], inst["p"], inst["dt"], inst["ref"].shape[0] - 1
    # dynamics by the kinematics, terminal, objective term by term
    for k in range(H):
        assert np.allclose(x[k + 1], kin_step(x[k], u[k], m, g, dt), atol=1e-10)
    assert np.allclose(x[H], inst["ref"][H], atol=1e-10)
    assert abs(objective(inst, x, u) - r["obj"]) <= 1e-10 * (1 + abs(r["obj"]))
    # every segment's curve: derivatives within the bounds, positions on the
    # node side of the plane (dense sampling; the convex-hull property)
    t = np.linspace(0, 1, 201)
    for k in range(H):
        P = segment_control_points(inst, x, k)
        pts = bezier_points(P, t)
        h, l = inst["planes"][k, :m], inst["planes"][k, m]
        assert np.all(pts @ h >= l - 1e-9)
        if inst["keepin_A"] is not None:
            assert np.all(pts @ inst["keepin_A"].T <= inst["keepin_b"] + 1e-9)
        for d in range(1, g + 1):
            Dd = P.copy()
            for _ in range(d):
                Dd = (Dd[1:] - Dd[:-1]) * (Dd.shape[0] - 1) / dt
            vals = bezier_points(Dd, t) if Dd.shape[0] > 1 else np.repeat(Dd, len(t), axis=0)
            assert np.abs(vals).max() <= inst["bounds"][d - 1] + 1e-9
    # KKT by non-negative least squares
    qp = r["qp"]
    kk = mpc.kkt_residuals(qp["P"], qp["q"], qp["Aeq"], qp["beq"], qp["Ain"], qp["bin"], r["z"])
    assert kk["eq"] < 1e-10 and kk["viol"] < 1e-10 and kk["stat"] < 1e-8 * (1 + kk["grad"])


def test_active_constraints_bind():
    """Planes cutting into the reference make some safety rows active, and the
    solution differs from the unconstrained one."""
    inst = instance(4)
    m = inst["m"]
    for k in (2, 5):
        inst["planes"][k, m] += 0.015         # the plane now cuts into the reference segment
    r = solve(inst)
    assert r["status"] == mpc.OK and len(r["active"]) > 0
    free = dict(inst, planes=np.zeros_like(inst["planes"]))
    r0 = solve(free)
    assert np.abs(r["x"] - r0["x"]).max() > 1e-3


@pytest.mark.parametrize("m,g,p", [(2, 2, 5), (3, 3, 7)])
def test_unconstrained_mpc_equals_condensed_least_squares(m, g, p):
    """No planes and bounds far away: the optimum of the equality-constrained
    least-squares problem in the inputs alone (states written as
    x_k = (kinematics of x0 and u_0..u_{k-1}), terminal equality through the
    null space)."""
    inst = instance(5, m=m, g=g, p=p, H=6, planes_on=False, bounds=(1e6, 1e6, 1e6))
    r = solve(inst)
    n, H, dt = m * g, 6, inst["dt"]
    nu = m * H
    # x_k as an affine function of u, by simulating unit inputs with the kinematics
    def traj(uvec):
        xs = [inst["x0"]]
        for k in range(H):
            xs.append(kin_step(xs[-1], uvec[k * m:(k + 1) * m], m, g, dt))
        return np.array(xs)
    X0 = traj(np.zeros(nu))
    G = np.stack([traj(np.eye(nu)[j]) - X0 for j in range(nu)], axis=-1)   # [H+1][n][nu]
    rows, rhs = [], []
    for k in range(H):
        w = np.sqrt(inst["Q"])
        rows.append(w[:, None] * G[k]); rhs.append(w * (inst["ref"][k] - X0[k]))
        w = np.sqrt(inst["F"])
        rows.append(w[:, None] * (G[k + 1] - G[k])); rhs.append(-w * (X0[k + 1] - X0[k]))
        w = np.sqrt(inst["R"])
        S = np.zeros((m, nu)); S[:, k * m:(k + 1) * m] = np.eye(m)
        rows.append(w[:, None] * S); rhs.append(np.zeros(m))
    w = np.sqrt(inst["V"])
    rows.append(w[:, None] * G[H]); rhs.append(w * (inst["ref"][H] - X0[H]))
    M, y = np.concatenate(rows), np.concatenate(rhs)
    # terminal equality G_H u = r_H - X0_H: u = u_p + N v
    E, e = G[H], inst["ref"][H] - X0[H]
    u_p = np.linalg.lstsq(E, e, rcond=None)[0]
    _, sv, Vt = np.linalg.svd(E)
    Nsp = Vt[np.sum(sv > 1e-12 * sv[0]):].T
    v = np.linalg.lstsq(M @ Nsp, y - M @ u_p, rcond=None)[0]
    u = (u_p + Nsp @ v).reshape(H, m)
    assert np.allclose(r["u"], u, atol=1e-8 * (1 + np.abs(u).max()))


def test_planted_mistakes_are_caught():
    inst = instance(6)
    r = solve(inst)
    x, u = r["x"], r["u"]
    # dropping the path-length term from the assembled objective, or the
    # input term, changes the term-by-term objective check
    for drop in ("F", "R"):
        bad = dict(inst, **{drop: np.zeros_like(inst[drop])})
        assert abs(objective(bad, x, u) - r["obj"]) > 1e-6
    # a plane with its sign flipped puts the solution on the wrong side
    m = inst["m"]
    flipped = inst["planes"].copy()
    flipped[:, :m] *= -1
    flipped[:, m] *= -1
    t = np.linspace(0, 1, 51)
    bad_side = False
    for k in range(inst["ref"].shape[0] - 1):
        pts = bezier_points(segment_control_points(inst, x, k), t)
        bad_side |= bool(np.any(pts @ flipped[k, :m] < flipped[k, m] - 1e-9))
    assert bad_side
    # transposed state layout (axis-major instead of derivative-major) breaks the dynamics check
    xt = x.reshape(x.shape[0], inst["g"], m).transpose(0, 2, 1).reshape(x.shape[0], -1)
    assert not np.allclose(xt[1], kin_step(xt[0], u[0], m, inst["g"], inst["dt"]), atol=1e-6)


def test_infeasible_mpc():
    inst = instance(7)
    m = inst["m"]
    inst["planes"][3, :m] = [1.0, 0.0]
    inst["planes"][3, m] = 1e3            # every point must have z_0 >= 1000
    assert solve(inst)["status"] == mpc.INFEASIBLE


@pytest.mark.parametrize("seed,m,g,p", [(1, 2, 2, 5), (2, 2, 2, 5), (4, 3, 3, 7), (5, 3, 3, 7)])
def test_optimum_is_no_worse_than_the_feasible_reference(seed, m, g, p):
    """The reference trajectory (its nodes and the inputs that produce them)
    satisfies every row, so the optimum's objective cannot exceed its own --
    a check of optimality that does not use the solver's multipliers."""
    inst = instance(seed, m=m, g=g, p=p)
    r = solve(inst)
    assert r["status"] == mpc.OK
    qp = r["qp"]
    H = inst["ref"].shape[0] - 1
    A, B = mpc.discretize(m, g, inst["dt"])
    u_ref = np.array([np.linalg.lstsq(B, inst["ref"][k + 1] - A @ inst["ref"][k], rcond=None)[0] for k in range(H)])
    z_ref = np.concatenate([inst["ref"][1:].reshape(-1), u_ref.reshape(-1)])
    assert np.abs(qp["Aeq"] @ z_ref - qp["beq"]).max() < 1e-10
    assert (qp["Ain"] @ z_ref - qp["bin"]).max() <= 1e-12
    assert r["obj"] <= objective(inst, inst["ref"], u_ref) + 1e-12

