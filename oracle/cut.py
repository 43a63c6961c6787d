"""FP64 oracle of the keep-out cut (Sec. III-B, Algorithm 2, Cut-QP).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For an edge (i, j) and a duration T the position control points P_0..P_p of
its curve are P_l = (sum_c D[l][c] xL_c) + (sum_c D[l][g+c] xR_c) per axis
(halves summed left to right, no FMA: the canonical order of the edge build).
An obstacle O = {z : A z <= b} (convex polytope, Assumption 1) is hit when the
convex hull of the control points meets O (Property 1 makes a miss of the hull
sufficient for a collision-free curve).  With G[l][r] = A_r . P_l - b_r
(summed left to right over the axes, then b subtracted):

  1. some control point lies in O (every row G[l][r] <= 0)       -> hit;
  2. some facet r has every control point strictly outside (G[l][r] > 0 for
     all l): a separating hyperplane                               -> miss;
  3. otherwise the Cut-QP's answer, read as the linear programme it decides:
        delta* = min over lambda in the simplex of max_r (G^T lambda)_r,
     the hull meets O iff delta* <= 0 (touching counts as a hit, as the
     inclusive inequalities of Theorem 1 and of the Cut-QP do).

Step 3 is solved exactly: the FP64 values of G are taken as exact rationals
and the matrix game is solved by the simplex method in fractions.Fraction with
Bland's rule (shifted payoffs M = G + c > 0, max 1^T u s.t. M^T u <= 1, u >= 0,
value = 1 / max - c).  The solution carries certificates: the mixing weights
lambda (a hull point in O when delta* <= 0) and the row weights y (a separating
hyperplane sum_r y_r A_r when delta* > 0).

An (edge, T) survives when its curve misses every obstacle; an edge survives
with the durations that survive, its weight the minimum cost over them (ties to
the lowest duration index).
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Optional, Tuple

import numpy as np


def control_points(D: np.ndarray, g: int, m: int, xi: np.ndarray, xj: np.ndarray) -> np.ndarray:
    """Position control points [p+1][m] in the canonical FP64 order."""
    p1 = D.shape[0]
    P = np.zeros((p1, m))
    for l in range(p1):
        for a in range(m):
            sl = 0.0
            for c in range(g):
                sl = sl + D[l][c] * xi[c * m + a]
            sr = 0.0
            for c in range(g):
                sr = sr + D[l][g + c] * xj[c * m + a]
            P[l, a] = sl + sr
    return P


def margins(P: np.ndarray, A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """G[l][r] = A_r . P_l - b_r, axes summed left to right, then b subtracted."""
    G = np.zeros((P.shape[0], A.shape[0]))
    for l in range(P.shape[0]):
        for r in range(A.shape[0]):
            s = 0.0
            for a in range(P.shape[1]):
                s = s + A[r, a] * P[l, a]
            G[l, r] = s - b[r]
    return G


def game_value(G: np.ndarray) -> Tuple[Fraction, List[Fraction], List[Fraction]]:
    """Exact value of min_lambda max_r (G^T lambda)_r over the simplex, with
    the optimal lambda (over rows l) and y (over columns r)."""
    nl, nr = G.shape
    Gf = [[Fraction(float(G[l, r])) for r in range(nr)] for l in range(nl)]
    c = 1 - min(min(row) for row in Gf)          # shift: every payoff >= 1
    M = [[Gf[l][r] + c for r in range(nr)] for l in range(nl)]
    # tableau rows r: sum_l M[l][r] u_l + s_r = 1 ; columns: u_0..u_{nl-1}, s_0..s_{nr-1}, rhs
    nv = nl + nr
    tab = [[M[l][r] for l in range(nl)] + [Fraction(1 if k == r else 0) for k in range(nr)] + [Fraction(1)]
           for r in range(nr)]
    basis = [nl + r for r in range(nr)]
    obj = [Fraction(1)] * nl + [Fraction(0)] * nr   # maximise sum u
    while True:
        # reduced costs: obj_j - sum_r obj_basis[r] * tab[r][j]
        red = []
        for j in range(nv):
            rc = obj[j] - sum(obj[basis[r]] * tab[r][j] for r in range(nr))
            red.append(rc)
        enter = next((j for j in range(nv) if red[j] > 0), None)   # Bland: lowest index
        if enter is None:
            break
        best, leave = None, None
        for r in range(nr):
            if tab[r][enter] > 0:
                ratio = tab[r][nv] / tab[r][enter]
                if best is None or ratio < best or (ratio == best and basis[r] < basis[leave]):
                    best, leave = ratio, r
        assert leave is not None, "unbounded (cannot happen: M > 0)"
        pv = tab[leave][enter]
        tab[leave] = [v / pv for v in tab[leave]]
        for r in range(nr):
            if r != leave and tab[r][enter] != 0:
                f = tab[r][enter]
                tab[r] = [a - f * bb for a, bb in zip(tab[r], tab[leave])]
        basis[leave] = enter
    u = [Fraction(0)] * nv
    for r in range(nr):
        u[basis[r]] = tab[r][nv]
    z = sum(u[:nl])
    value = 1 / z - c
    lam = [v / z for v in u[:nl]]
    # dual: y_r = reduced-cost multipliers of the slacks (-red of s_r), scaled to the simplex
    ysh = [sum(obj[basis[k]] * tab[k][nl + r] for k in range(nr)) for r in range(nr)]
    ys = sum(ysh)
    y = [v / ys for v in ysh]
    return value, lam, y


def obstacle_hit(G: np.ndarray) -> Tuple[bool, int, Optional[Fraction]]:
    """(hit, step that decided it (1, 2 or 3), exact delta* when step 3)."""
    if np.any(np.all(G <= 0.0, axis=1)):
        return True, 1, None
    if np.any(np.all(G > 0.0, axis=0)):
        return False, 2, None
    v, _, _ = game_value(G)
    return v <= 0, 3, v


def cut(op, csr_detail: dict, obst_off, A_o, b_o) -> dict:
    """Cut of an oracle graph (OracleProblem.csr(with_detail=True)) against
    obstacles given as CSR polytopes.  Returns the new CSR and per-step counts."""
    g, m, p = op.gamma, op.m, op.p
    n = op.n
    X = op.states
    off = np.asarray(obst_off, dtype=np.int64)
    A_o = np.asarray(A_o, dtype=np.float64).reshape(-1, m)
    b_o = np.asarray(b_o, dtype=np.float64)
    e = csr_detail["all"]
    keep = e["mask"] != 0
    I, J, Mk, C = e["i"][keep], e["j"][keep], e["mask"][keep], e["costs"][keep]
    order = np.lexsort((J, I))
    I, J, Mk, C = I[order], J[order], Mk[order], C[order]
    steps = {1: 0, 2: 0, 3: 0}
    deltas = []
    rows_col, rows_w, rows_t, rows_m, rows_i = [], [], [], [], []
    for idx in range(len(I)):
        i, j, mask = int(I[idx]), int(J[idx]), int(Mk[idx])
        newmask = 0
        for t in range(op.nT):
            if not (mask >> t) & 1:
                continue
            P = control_points(op.D[t], g, m, X[i], X[j])
            ok = True
            for o in range(len(off) - 1):
                G = margins(P, A_o[off[o]:off[o + 1]], b_o[off[o]:off[o + 1]])
                hit, st, v = obstacle_hit(G)
                steps[st] += 1
                if v is not None:
                    deltas.append(float(v))
                if hit:
                    ok = False
                    break
            if ok:
                newmask |= 1 << t
        if newmask:
            costs = C[idx]
            best = min((t for t in range(op.nT) if (newmask >> t) & 1), key=lambda t: (costs[t], t))
            rows_i.append(i)
            rows_col.append(j)
            rows_m.append(newmask)
            rows_w.append(costs[best])
            rows_t.append(best)
    N = op.N
    cnt = np.bincount(np.asarray(rows_i, dtype=np.int64), minlength=N)
    row_off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    return {"row_off": row_off, "col": np.asarray(rows_col, dtype=np.int32), "w": np.asarray(rows_w),
            "t": np.asarray(rows_t, dtype=np.uint8), "mask": np.asarray(rows_m, dtype=np.uint32),
            "steps": steps, "deltas": np.asarray(deltas)}
