"""Independent checks ("pins") for the oracle's coefficient tables and pair test.

Every check here reaches its expected value by a route other than the
oracle's: textbook closed forms (cubic / quintic Hermite in Bezier form),
direct expansion of the Bernstein polynomial into the power basis followed by
numpy differentiation, the textbook hodograph of a Bezier curve (differences
of control points), and brute-force evaluation of the inequalities.  Each
function returns the largest relative violation it found, so a test can both
assert that the oracle passes and that a deliberately broken table fails.
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np
from numpy.polynomial import polynomial as npoly


def bernstein_to_power(P: np.ndarray) -> np.ndarray:
    """Power-basis coefficients (in u) of sum_l P_l C(p,l) u^l (1-u)^(p-l); P is [p+1][...]."""
    p = P.shape[0] - 1
    out = np.zeros_like(P, dtype=np.float64)
    for l in range(p + 1):
        for k in range(p - l + 1):
            out[l + k] += P[l] * comb(p, l) * comb(p - l, k) * (-1.0) ** k
    return out


def eval_bernstein(P: np.ndarray, u: np.ndarray) -> np.ndarray:
    """de Casteljau evaluation of a scalar Bezier curve at parameters u."""
    pts = np.repeat(np.asarray(P, dtype=np.float64)[None, :], u.shape[0], axis=0)
    uu = u[:, None]
    for r in range(pts.shape[1] - 1, 0, -1):
        pts = (1.0 - uu) * pts[:, :r] + uu * pts[:, 1:r + 1]
    return pts[:, 0]


def t_derivative_at(P: np.ndarray, T: float, c: int, u: np.ndarray) -> np.ndarray:
    """d^c/dt^c of the Bezier curve with control points P at u = t/T (power basis + polyder)."""
    pw = bernstein_to_power(P)
    d = npoly.polyder(pw, c) if c else pw
    return npoly.polyval(u, d) / T ** c


def textbook_hermite(gamma: int, T: float, xi: np.ndarray) -> np.ndarray:
    """Closed-form minimal-degree Hermite control points (one axis).

    gamma = 2 (cubic):  P0 = x0, P1 = x0 + T v0/3, P2 = x1 - T v1/3, P3 = x1.
    gamma = 3 (quintic): P0 = x0, P1 = x0 + T v0/5, P2 = x0 + 2T v0/5 + T^2 a0/20,
                         P3 = x1 - 2T v1/5 + T^2 a1/20, P4 = x1 - T v1/5, P5 = x1.
    """
    if gamma == 2:
        x0, v0, x1, v1 = xi
        return np.array([x0, x0 + T * v0 / 3, x1 - T * v1 / 3, x1])
    if gamma == 3:
        x0, v0, a0, x1, v1, a1 = xi
        return np.array([x0, x0 + T * v0 / 5, x0 + 2 * T * v0 / 5 + T * T * a0 / 20,
                         x1 - 2 * T * v1 / 5 + T * T * a1 / 20, x1 - T * v1 / 5, x1])
    raise ValueError("closed form only for gamma 2, 3")


def elevate(P: np.ndarray, r: int) -> np.ndarray:
    """Textbook degree elevation by r: P'_i = sum_j C(q,j) C(r,i-j) / C(q+r,i) P_j."""
    q = P.shape[0] - 1
    out = np.zeros(q + r + 1)
    for i in range(q + r + 1):
        for j in range(max(0, i - r), min(q, i) + 1):
            out[i] += comb(q, j) * comb(r, i - j) / comb(q + r, i) * P[j]
    return out


def _rand_xi(rng, gamma, scale=1.0):
    return rng.uniform(-scale, scale, 2 * gamma)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / (1.0 + np.abs(b))))


def pin_endpoints(gamma, p, T, D, rng, trials=8):
    """b^(c)(0) = xL_c and b^(c)(T) = xR_c for c < gamma (Lemma 1)."""
    worst = 0.0
    u = np.array([0.0, 1.0])
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        P = D @ xi
        for c in range(gamma):
            v = t_derivative_at(P, T, c, u)
            worst = max(worst, _rel(v, [xi[c], xi[gamma + c]]))
    return worst


def pin_minimal_degree(gamma, T, D, rng, trials=8):
    """At p = 2g-1 the control points equal the textbook Hermite-Bezier closed form."""
    worst = 0.0
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        worst = max(worst, _rel(D @ xi, textbook_hermite(gamma, T, xi)))
    return worst


def pin_elevation(gamma, p, T, D, rng, trials=4, samples=1025):
    """The degree-p curve is the minimal Hermite curve, elevated (same b(t) everywhere)."""
    worst = 0.0
    u = np.linspace(0.0, 1.0, samples)
    q = 2 * gamma - 1
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        ref = textbook_hermite(gamma, T, xi) if gamma in (2, 3) else None
        P = D @ xi
        if ref is not None:
            worst = max(worst, _rel(P, elevate(ref, p - q)))
            worst = max(worst, _rel(eval_bernstein(P, u), eval_bernstein(ref, u)))
    return worst


def pin_hodograph(gamma, p, T, D, H, rng, trials=6, samples=65):
    """Reach rows of order k are the degree p-k control points of b^(k)(t):
    sum_j Q_j B_j^{p-k}(u) equals the k-th t-derivative of the curve D xi, and
    Q_j equals the textbook hodograph p!/(p-k)! T^-k Delta^k P_j."""
    worst = 0.0
    u = np.linspace(0.0, 1.0, samples)
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        P = D @ xi
        row = 0
        for k in range(1, gamma + 1):
            Q = H[row:row + p - k + 1] @ xi
            row += p - k + 1
            dk = P.copy()
            for _ in range(k):
                dk = np.diff(dk)
            hod = factorial(p) / factorial(p - k) / T ** k * dk
            worst = max(worst, _rel(Q, hod))
            worst = max(worst, _rel(eval_bernstein(Q, u), t_derivative_at(P, T, k, u)))
    return worst


def pin_cost_rows(gamma, p, T, D, C, rng, trials=6, samples=65):
    """Cost rows are consecutive differences of the degree-p control points of
    b^(d)(t), d = 0..g-1 (rows of the state-space matrix P of Eq. BezDef)."""
    worst = 0.0
    u = np.linspace(0.0, 1.0, samples)
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        P = D @ xi
        for d in range(gamma):
            diffs = C[d] @ xi
            W = np.concatenate([[xi[d]], xi[d] + np.cumsum(diffs)])   # W_0 = b^(d)(0) = xL_d
            worst = max(worst, _rel(eval_bernstein(W, u), t_derivative_at(P, T, d, u)))
    return worst


def energy(P: np.ndarray, T: float, k: int) -> float:
    """int_0^T |b^(k)(t)|^2 dt by Gauss-Legendre quadrature, exact for the
    polynomial degree of the integrand (numpy's derivative of the power form)."""
    deg = len(P) - 1
    npts = max(1, deg - k + 1)
    x, w = np.polynomial.legendre.leggauss(npts)
    u = 0.5 * (x + 1.0)
    v = t_derivative_at(P, T, k, u)
    return float(0.5 * T * np.sum(w * v * v))


def pin_minsnap_optimal(gamma, p, T, D, rng, trials=6):
    """Minimum-energy interior points: every interior control point is at a
    stationary point of int |b^(g+1)|^2 (central difference of the energy is
    zero to first order, curvature positive), and the energy is at most that
    of the elevated minimal-degree curve with the same end conditions."""
    worst = 0.0
    k = gamma + 1
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        P = D @ xi
        J0 = energy(P, T, k)
        scale = max(J0, 1e-300)
        for l in range(gamma, p - gamma + 1):
            h = 1e-3 * (1.0 + abs(P[l]))
            Pp, Pm = P.copy(), P.copy()
            Pp[l] += h
            Pm[l] -= h
            Jp, Jm = energy(Pp, T, k), energy(Pm, T, k)
            curv = Jp + Jm - 2 * J0
            assert curv > 0
            worst = max(worst, abs(Jp - Jm) / curv)   # 0 at the minimiser (J is exactly quadratic)
        if gamma in (2, 3):
            ref = elevate(textbook_hermite(gamma, T, xi), p - (2 * gamma - 1))
            worst = max(worst, max(0.0, J0 - energy(ref, T, k)) / scale)
    return worst


def pin_minsnap_natural(gamma, p, T, D, rng, trials=6):
    """At p = 2g+1 the minimiser has b^(g+1) = 0 at both ends (the natural
    boundary conditions of the variational problem; for g = 1 this makes the
    cubic a straight line: P_l = xL + l (xR - xL) / 3)."""
    worst = 0.0
    if p != 2 * gamma + 1:
        return worst
    for _ in range(trials):
        xi = _rand_xi(rng, gamma, 3.0)
        P = D @ xi
        ends = t_derivative_at(P, T, gamma + 1, np.array([0.0, 1.0]))
        mid = t_derivative_at(P, T, gamma + 1, np.linspace(0.0, 1.0, 9))
        worst = max(worst, float(np.max(np.abs(ends))) / max(1.0, float(np.max(np.abs(mid)))))
        if gamma == 1:
            line = xi[0] + np.arange(p + 1) / p * (xi[1] - xi[0])
            worst = max(worst, _rel(P, line))
    return worst


def all_table_pins(gamma, p, T, tb, seed=0, interior="elevate"):
    rng = np.random.default_rng(seed)
    res = {"endpoints": pin_endpoints(gamma, p, T, tb["D"], rng),
           "hodograph": pin_hodograph(gamma, p, T, tb["D"], tb["H"], rng),
           "cost_rows": pin_cost_rows(gamma, p, T, tb["D"], tb["C"], rng)}
    if interior == "minsnap" and p > 2 * gamma - 1:
        res["minsnap_optimal"] = pin_minsnap_optimal(gamma, p, T, tb["D"], rng)
        res["minsnap_natural"] = pin_minsnap_natural(gamma, p, T, tb["D"], rng)
    else:
        res["elevation"] = pin_elevation(gamma, p, T, tb["D"], rng)
    if p == 2 * gamma - 1:
        res["minimal"] = pin_minimal_degree(gamma, T, tb["D"], rng)
    return res


# ---------------------------------------------------------------------------
# Brute-force pair test on tiny inputs, written from the definitions with
# textbook Bezier identities only (no reach/cost table).
# ---------------------------------------------------------------------------

def brute_pair(m, gamma, p, bounds, T, D, A, b, xi_state, xj_state, cost_mode="state"):
    """Feasibility margin and cost of one (pair, T) from control points alone.

    Returns (reach_margin, free_margin, cost): reach_margin = min over k, axes
    and hodograph control points of c_k - |Q|; free_margin = min over rows and
    control points of b - A P; cost = sum_l ||Pstate_{l+1} - Pstate_l||.
    """
    pts = np.zeros((p + 1, m))
    for a in range(m):
        xi = np.array([xi_state[c * m + a] for c in range(gamma)] + [xj_state[c * m + a] for c in range(gamma)])
        pts[:, a] = D @ xi
    rm = np.inf
    for k in range(1, gamma + 1):
        dk = pts.copy()
        for _ in range(k):
            dk = np.diff(dk, axis=0)
        Q = factorial(p) / factorial(p - k) / T ** k * dk
        rm = min(rm, float(np.min(bounds[k - 1] - np.abs(Q))))
    fm = float(np.min(b[:, None] - A @ pts.T)) if A.shape[0] else np.inf
    # state-space control points: degree-p representation of b^(d) (hodograph elevated by d)
    rows = []
    for d in range(gamma if cost_mode == "state" else 1):
        dk = pts.copy()
        for _ in range(d):
            dk = np.diff(dk, axis=0)
        Qd = factorial(p) / factorial(p - d) / T ** d * dk
        rows.append(np.stack([elevate(Qd[:, a], d) for a in range(m)], axis=1))
    S = np.concatenate(rows, axis=1)
    cost = float(np.sum(np.linalg.norm(np.diff(S, axis=0), axis=1)))
    return rm, fm, cost
