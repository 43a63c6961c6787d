"""FP64 oracle of the MPC refinement step (Sec. III-D, Eq. (MPC) with its
dynamics, initial-condition, safety, input and terminal constraints; the
paper solves it repeatedly in an SQP fashion, each time with the separating
planes of the current iterate).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The problem, written out in the paper's variables (the horizon is H, the
step dt; the state x in R^n, n = m g, is stored derivative-major as in the
graph: x = [x^(0) (m), x^(1) (m), ..., x^(g-1) (m)], the input u in R^m is the
g-th derivative of every axis):

  min  sum_{k=0}^{H-1} (x_k - r_k)' Q (x_k - r_k) + (x_{k+1} - x_k)' F (x_{k+1} - x_k)
                       + u_k' R u_k   +   (x_H - r_H)' V (x_H - r_H)
  s.t. x_{k+1} = A x_k + B u_k                         (exact discretisation)
       x_0 = the measured state                         (zero tracking-error set)
       |H_r xi_{k,a}| <= c_{ord(r)}  for every reach row r of duration dt,
            axis a and segment k (Theorem 1 on the boundary conditions
            xi_{k,a} = [x_k^(0..g-1)_a ; x_{k+1}^(0..g-1)_a])
       h_k . P_l(k) >= l_k  for every control point P_l(k) = D xi_k of
            segment k (l = 1..p for k = 0, whose P_0 is the fixed x_0; 0..p
            otherwise), with (h_k, l_k) the separating plane of node k and its
            nearest obstacle (adjacentHyperplane); no rows when h_k = 0
       A_d P_l(k) <= b_d  for the same control points (keep-in polytope, optional)
       x_H = r_H                                        (terminal)

Q, F, V are diagonal with positive entries in R^n and R in R^m (the paper
allows symmetric positive definite matrices; diagonal weights are the
restriction taken here).  Every weight positive makes the objective strictly
convex in z = [x_1..x_H, u_0..u_{H-1}], so the optimum is unique.

Solution method (independent of the GPU path, which condenses the states away
and runs a dual active-set method): this module keeps the states as
variables with the dynamics as equality rows, finds a feasible point with a
linear program (scipy's HiGHS, a library step), and then runs the textbook
primal active-set method for convex QPs: solve the equality-constrained
subproblem on the working set; a zero step with non-negative multipliers is
optimal, a zero step with a negative multiplier drops that constraint, a
non-zero step goes as far as the first blocking constraint and adds it
(rules in solve_qp).  The inequality rows are kept once each (a reach row
of a boundary derivative is the same row in the two segments that share the
node).
"""
from __future__ import annotations

from math import factorial
from typing import Dict, Optional

import numpy as np
from scipy.linalg import expm
from scipy.optimize import linprog, nnls

from oracle import tables as OT

OK, INFEASIBLE, MAXITER = 0, 1, 2


def discretize(m: int, g: int, dt: float):
    """Exact zero-order-hold discretisation of the chain of integrators
    (each axis: g states, input the g-th derivative) in the derivative-major
    layout: the matrix exponential of the augmented continuous system
    [[Ac, Bc], [0, 0]] dt (Van Loan), a library step."""
    n = m * g
    M = np.zeros((n + m, n + m))
    for a in range(m):
        for c in range(g - 1):
            M[c * m + a, (c + 1) * m + a] = 1.0
        M[(g - 1) * m + a, n + a] = 1.0
    E = expm(M * dt)
    return E[:n, :n], E[:n, n:]


def build_qp(m: int, g: int, p: int, bounds, dt: float, x0, ref, planes, Q, F, R, V,
             keepin_A=None, keepin_b=None, interior: str = "elevate") -> Dict[str, np.ndarray]:
    """The QP in z = [x_1 .. x_H (n each), u_0 .. u_{H-1} (m each)]:
    minimise 1/2 z'Pz + q'z + const subject to Aeq z = beq, Ain z <= bin.
    planes: [H][m+1] (h, l) per segment; ref: [H+1][n]."""
    n = m * g
    x0 = np.asarray(x0, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    planes = np.asarray(planes, dtype=np.float64)
    H = ref.shape[0] - 1
    nz = n * H + m * H
    Q, F, R, V = (np.asarray(w, dtype=np.float64) for w in (Q, F, R, V))
    A, B = discretize(m, g, dt)
    tab = OT.tables(g, p, [dt], interior)
    D, Hr = tab["D"][0], tab["H"][0]
    orders = OT.reach_row_orders(g, p)

    def xs(k):   # z-slice of x_k (k >= 1)
        return slice(n * (k - 1), n * k)

    def us(k):
        return slice(n * H + m * k, n * H + m * (k + 1))

    # objective: every term (Sx z + s0)' W (Sx z + s0) with W diagonal
    P = np.zeros((nz, nz))
    q = np.zeros(nz)
    const = 0.0

    def add_term(S, s0, W):
        nonlocal const, P, q
        P += 2.0 * S.T @ (W[:, None] * S)
        q += 2.0 * S.T @ (W * s0)
        const += float(s0 @ (W * s0))

    def sel_x(k):
        """(S, s0) with x_k = S z + s0."""
        S = np.zeros((n, nz))
        if k == 0:
            return S, x0.copy()
        S[:, xs(k)] = np.eye(n)
        return S, np.zeros(n)

    for k in range(H):
        S, s0 = sel_x(k)
        add_term(S, s0 - ref[k], Q)
        S1, s1 = sel_x(k + 1)
        add_term(S1 - S, s1 - s0, F)
        Su = np.zeros((m, nz))
        Su[:, us(k)] = np.eye(m)
        add_term(Su, np.zeros(m), R)
    S, s0 = sel_x(H)
    add_term(S, s0 - ref[H], V)

    # equalities: dynamics, terminal
    Aeq, beq = [], []
    for k in range(H):
        S0, c0 = sel_x(k)
        S1, c1 = sel_x(k + 1)
        Su = np.zeros((n, nz))
        Su[:, us(k)] = B
        rows = S1 - A @ S0 - Su                    # x_{k+1} - A x_k - B u_k = 0
        Aeq.append(rows)
        beq.append(A @ c0 - c1)
    S, c = sel_x(H)
    Aeq.append(S)
    beq.append(ref[H] - c)
    Aeq = np.concatenate(Aeq)
    beq = np.concatenate(beq)

    # inequalities
    Ain, bin_ = [], []
    for k in range(H):
        S0, c0 = sel_x(k)
        S1, c1 = sel_x(k + 1)
        for a in range(m):
            # xi_{k,a} = T_a z + t_a
            T = np.concatenate([S0[[cc * m + a for cc in range(g)]], S1[[cc * m + a for cc in range(g)]]])
            t = np.concatenate([c0[[cc * m + a for cc in range(g)]], c1[[cc * m + a for cc in range(g)]]])
            for r in range(Hr.shape[0]):
                cb = float(bounds[orders[r] - 1])
                row, off = Hr[r] @ T, float(Hr[r] @ t)
                Ain.append(row)
                bin_.append(cb - off)
                Ain.append(-row)
                bin_.append(cb + off)
        # control points of segment k: P_l = Cp_l z + cp_l  [p+1][m]
        Cp = np.zeros((p + 1, m, nz))
        cp = np.zeros((p + 1, m))
        for a in range(m):
            T = np.concatenate([S0[[cc * m + a for cc in range(g)]], S1[[cc * m + a for cc in range(g)]]])
            t = np.concatenate([c0[[cc * m + a for cc in range(g)]], c1[[cc * m + a for cc in range(g)]]])
            Cp[:, a, :] = D @ T
            cp[:, a] = D @ t
        h, l = planes[k, :m], planes[k, m]
        first = 1 if k == 0 else 0
        if np.any(h != 0.0):
            for li in range(first, p + 1):          # -h . P_l <= -l
                Ain.append(-(h @ Cp[li]))
                bin_.append(-l + float(h @ cp[li]))
        if keepin_A is not None:   # P_0 of segment k is P_p of segment k-1 (or the fixed x_0)
            KA = np.asarray(keepin_A, dtype=np.float64).reshape(-1, m)
            Kb = np.asarray(keepin_b, dtype=np.float64)
            for li in range(1, p + 1):
                for r in range(KA.shape[0]):
                    Ain.append(KA[r] @ Cp[li])
                    bin_.append(Kb[r] - float(KA[r] @ cp[li]))
    Ain = np.array(Ain) if Ain else np.zeros((0, nz))
    bin_ = np.array(bin_) if bin_ else np.zeros(0)
    # a constraint met twice (the reach row of a derivative that is a boundary
    # condition, at the node two segments share) is kept once
    if Ain.shape[0]:
        _, first_idx = np.unique(np.concatenate([Ain, bin_[:, None]], axis=1), axis=0, return_index=True)
        keep = np.sort(first_idx)
        Ain, bin_ = Ain[keep], bin_[keep]
    return {"P": P, "q": q, "const": const, "Aeq": Aeq, "beq": beq, "Ain": Ain, "bin": bin_,
            "H": H, "n": n, "m": m}


def _independent(rows: np.ndarray, cand, base, tol=1e-10):
    """Greedy: add candidate rows that keep [base; chosen] of full row rank."""
    chosen = list(base)
    for i in cand:
        M = rows[chosen + [i]]
        if np.linalg.matrix_rank(M, tol=tol * max(1.0, np.abs(M).max())) == len(chosen) + 1:
            chosen.append(i)
    return chosen[len(base):]


def solve_qp(P, q, Aeq, beq, Ain, bin_, max_iter: int = 20000, z0: Optional[np.ndarray] = None):
    """Convex QP min 1/2 z'Pz + q'z s.t. Aeq z = beq, Ain z <= bin (P positive
    definite).  Returns (status, z, working set of inequalities at the
    optimum, multipliers of the equalities, multipliers of that working set).

    Phase 1 (a library step): the feasible point of largest normalised slack
    t (at most 1), max t s.t. Ain z + |Ain_i| t <= bin, Aeq z = beq, so that
    usually no inequality is active where phase 2 starts.  Phase 2: the
    primal active-set method; the most negative multiplier leaves the working
    set and the first blocking row enters it, both on the lowest index among
    ties, and after 50 zero-length steps in a row the least index among the
    negative multipliers leaves instead (against cycling).  After a full
    unblocked step the point minimises the objective on the working set, so
    the next solve only supplies the multipliers (its step is rounding)."""
    nz = P.shape[0]
    ne, ni = Aeq.shape[0], Ain.shape[0]
    rown = np.linalg.norm(Ain, axis=1) if ni else np.zeros(0)
    if z0 is None:
        c = np.zeros(nz + 1)
        c[-1] = -1.0
        A_ub = np.concatenate([Ain, rown[:, None]], axis=1) if ni else None
        A_eq = np.concatenate([Aeq, np.zeros((ne, 1))], axis=1) if ne else None
        lp = linprog(c, A_ub=A_ub, b_ub=bin_ if ni else None, A_eq=A_eq, b_eq=beq if ne else None,
                     bounds=[(None, None)] * nz + [(0.0, 1.0)], method="highs")
        if lp.status == 2:
            return INFEASIBLE, None, [], None, None
        if lp.status != 0:
            raise RuntimeError(f"phase 1 failed: {lp.message}")
        z = lp.x[:nz].astype(np.float64)
    else:
        z = np.asarray(z0, dtype=np.float64).copy()

    def row_tol(i):
        return 1e-9 * (1.0 + abs(bin_[i]) + rown[i] * np.abs(z).max())

    act = [i for i in range(ni) if Ain[i] @ z - bin_[i] >= -row_tol(i)]
    allrows = np.concatenate([Aeq, Ain]) if ni else Aeq
    W = sorted(i - ne for i in _independent(allrows, [ne + i for i in act], list(range(ne))))
    zero_run = 0
    at_min = False      # z minimises the objective on the working set (a full step was just taken)
    for it in range(max_iter):
        AW = np.concatenate([Aeq, Ain[W]]) if W else Aeq
        k = AW.shape[0]
        K = np.zeros((nz + k, nz + k))
        K[:nz, :nz] = P
        K[:nz, nz:] = AW.T
        K[nz:, :nz] = AW
        grad = P @ z + q
        rhs = np.concatenate([-grad, np.zeros(k)])
        sol = np.linalg.solve(K, rhs)
        step, lam = sol[:nz], sol[nz:]      # P step + AW' lam = -(P z + q): lam are the multipliers
        # a zero step up to the solve's rounding: measured against the size of
        # the stationarity terms (gradient and A_W' lam), or negligible next to z
        gscale = 1.0 + np.abs(grad).max() + np.abs(AW.T @ lam).max()
        if at_min or np.abs(P @ step).max() <= 1e-11 * gscale or np.abs(step).max() <= 1e-10 * (1.0 + np.abs(z).max()):
            at_min = False
            mu = lam[ne:]
            neg = [j for j in range(len(W)) if mu[j] < -1e-10 * gscale]
            if not neg:
                return OK, z, list(W), lam[:ne], mu
            j = neg[0] if zero_run > 50 else min(neg, key=lambda jj: (mu[jj], jj))
            W = W[:j] + W[j + 1:]
            zero_run += 1
            continue
        # step length: first blocking inequality outside the working set; a row
        # the step runs along (a . step ~ 0) never blocks
        alpha, block = 1.0, -1
        if ni:
            ap = Ain @ step
            slack = bin_ - Ain @ z
            sn = np.linalg.norm(step)
            inW = set(W)
            for i in range(ni):
                if i in inW or ap[i] <= 1e-9 * rown[i] * sn:
                    continue
                t = max(slack[i], 0.0) / ap[i]
                if t < alpha:
                    alpha, block = t, i
        z = z + alpha * step
        zero_run = zero_run + 1 if alpha == 0.0 else 0
        if block >= 0:
            W = sorted(W + [block])
        else:
            at_min = True   # in exact arithmetic the next step on this working set is zero
    return MAXITER, z, list(W), None, None


def kkt_residuals(P, q, Aeq, beq, Ain, bin_, z, act_tol: float = 1e-8) -> Dict[str, float]:
    """Optimality check independent of the solver: primal feasibility,
    stationarity P z + q + Aeq' y + Ain_A' mu = 0 with mu >= 0 found by
    non-negative least squares over the inequalities active at z (the
    equality multipliers are split into two non-negative halves), and the
    residual of that fit."""
    nz = P.shape[0]
    scale = 1.0 + max(np.abs(beq).max(initial=0.0), np.abs(bin_).max(initial=0.0))
    eq = float(np.abs(Aeq @ z - beq).max(initial=0.0))
    viol = float(np.maximum(Ain @ z - bin_, 0.0).max(initial=0.0)) if Ain.shape[0] else 0.0
    act = np.where(Ain @ z - bin_ >= -act_tol * scale)[0] if Ain.shape[0] else np.zeros(0, dtype=int)
    Mt = np.concatenate([Aeq, -Aeq, Ain[act]]).T     # [nz][cols]
    grad = P @ z + q
    coef, res = nnls(Mt, -grad, maxiter=50 * Mt.shape[1] + 100)
    return {"eq": eq, "viol": viol, "stat": float(res), "grad": float(np.abs(grad).max()), "n_active": int(len(act))}


def mpc_qp(m, g, p, bounds, dt, x0, ref, planes, Q, F, R, V, keepin_A=None, keepin_b=None,
           interior: str = "elevate") -> Dict:
    """One QP of the refinement: node states x [H+1][n] (x_0 = x0), inputs
    u [H][m], the objective value (constants included) and the status."""
    qp = build_qp(m, g, p, bounds, dt, x0, ref, planes, Q, F, R, V, keepin_A, keepin_b, interior)
    st, z, W, y, mu = solve_qp(qp["P"], qp["q"], qp["Aeq"], qp["beq"], qp["Ain"], qp["bin"])
    H, n = qp["H"], qp["n"]
    if st != OK:
        return {"status": st, "qp": qp}
    x = np.concatenate([np.asarray(x0, dtype=np.float64)[None, :], z[:n * H].reshape(H, n)])
    u = z[n * H:].reshape(H, m)
    obj = 0.5 * float(z @ qp["P"] @ z) + float(qp["q"] @ z) + qp["const"]
    return {"status": OK, "x": x, "u": u, "obj": obj, "active": W, "qp": qp, "z": z}
