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
    """Position control points [p+1][m] in the canonical FP64 order: for every
    (l, a) at once, each half accumulated over c = 0..g-1 from 0.0 (numpy
    rounds every product and sum on its own), then the halves added."""
    xi = np.asarray(xi, dtype=np.float64).reshape(g, m)
    xj = np.asarray(xj, dtype=np.float64).reshape(g, m)
    sl = np.zeros((D.shape[0], m))
    sr = np.zeros((D.shape[0], m))
    for c in range(g):
        sl = sl + D[:, c:c + 1] * xi[c][None, :]
    for c in range(g):
        sr = sr + D[:, g + c:g + c + 1] * xj[c][None, :]
    return sl + sr


def margins(P: np.ndarray, A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """G[l][r] = A_r . P_l - b_r: for every (l, r) at once, the products over
    the axes a = 0..m-1 accumulated from 0.0, then b subtracted."""
    A = np.asarray(A, dtype=np.float64).reshape(-1, P.shape[1])
    s = np.zeros((P.shape[0], A.shape[0]))
    for a in range(P.shape[1]):
        s = s + P[:, a:a + 1] * A[None, :, a]
    return s - np.asarray(b, dtype=np.float64)[None, :]


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


def edge_decisions(G: np.ndarray, off: np.ndarray):
    """Algorithm 2 for one curve against every obstacle, in obstacle order,
    stopping at the first hit.  G holds the margins of all obstacles' rows
    side by side (obstacle o: columns off[o]..off[o+1]-1).  Returns (hit,
    per-step counts, exact delta* of every matrix game solved)."""
    steps = {1: 0, 2: 0, 3: 0}
    deltas = []
    for o in range(len(off) - 1):
        hit, st, v = obstacle_hit(G[:, off[o]:off[o + 1]])
        steps[st] += 1
        if v is not None:
            deltas.append(v)
        if hit:
            return True, steps, deltas
    return False, steps, deltas


def cut(op, csr_detail: dict, obst_off, A_o, b_o, rows=None) -> dict:
    """Cut of an oracle graph (OracleProblem.csr(with_detail=True)) against
    obstacles given as CSR polytopes, for the edges of the given rows (all by
    default).  Returns the new CSR (row offsets only when every row is cut),
    the kept edges' start vertices and per-duration costs (for comparisons),
    the per-step counts and the exact delta* of every game."""
    g, m = op.gamma, op.m
    X = op.states
    off = np.asarray(obst_off, dtype=np.int64)
    A_o = np.asarray(A_o, dtype=np.float64).reshape(-1, m)
    b_o = np.asarray(b_o, dtype=np.float64)
    e = csr_detail["all"]
    keep = e["mask"] != 0
    if rows is not None:
        keep &= np.isin(e["i"], np.asarray(rows))
    I, J, Mk, C = e["i"][keep], e["j"][keep], e["mask"][keep], e["costs"][keep]
    order = np.lexsort((J, I))
    I, J, Mk, C = I[order], J[order], Mk[order], C[order]
    steps = {1: 0, 2: 0, 3: 0}
    deltas = []
    out = {"i": [], "j": [], "w": [], "t": [], "mask": [], "costs": []}
    for idx in range(len(I)):
        i, j, mask = int(I[idx]), int(J[idx]), int(Mk[idx])
        newmask = 0
        for t in range(op.nT):
            if not (mask >> t) & 1:
                continue
            P = control_points(op.D[t], g, m, X[i], X[j])
            hit, st, dl = edge_decisions(margins(P, A_o, b_o), off)
            for k in steps:
                steps[k] += st[k]
            deltas += dl
            if not hit:
                newmask |= 1 << t
        if newmask:
            costs = C[idx]
            best = min((t for t in range(op.nT) if (newmask >> t) & 1), key=lambda t: (costs[t], t))
            out["i"].append(i)
            out["j"].append(j)
            out["mask"].append(newmask)
            out["w"].append(costs[best])
            out["t"].append(best)
            out["costs"].append(costs)
    N = op.N
    res = {"i": np.asarray(out["i"], dtype=np.int64), "j": np.asarray(out["j"], dtype=np.int32),
           "col": np.asarray(out["j"], dtype=np.int32), "w": np.asarray(out["w"], dtype=np.float64),
           "t": np.asarray(out["t"], dtype=np.int32), "mask": np.asarray(out["mask"], dtype=np.uint32),
           "costs": np.asarray(out["costs"], dtype=np.float64).reshape(-1, op.nT),
           "steps": steps, "deltas": np.asarray([float(d) for d in deltas])}
    if rows is None:
        cnt = np.bincount(res["i"], minlength=N)
        res["row_off"] = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    return res
