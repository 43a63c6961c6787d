"""Exact coefficient tables of the reachable Bezier polytope -- oracle side.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; it exists to check the CUDA path.

Every table maps the stacked boundary conditions of one axis,
xi = [xL_0 .. xL_{g-1}, xR_0 .. xR_{g-1}] (xL_c = c-th derivative of the start
state, xR_c of the end state, g = gamma), to a set of Bezier coefficients.
All arithmetic is exact (fractions.Fraction) and each entry is rounded to the
nearest double once, at the end, so a table entry is the correctly rounded
value of an exact rational function of T.

Route (chosen to be independent of the recurrences a GPU implementation would
use): the unique degree q = 2g-1 polynomial meeting the boundary conditions
(Lemma 1) is found in the monomial basis in u = t/T by exact Gaussian
elimination of the 2g x 2g Hermite system; it and its t-derivatives are then
converted to the Bernstein basis of the required degree with the identity
u^s = sum_{l>=s} C(l,s)/C(P,s) B_l^P(u).

Tables (per duration T):
  D  [(p+1)][2g]      control points of b(t) in degree p (Lemma 1; Sec. II-B);
                      for p > 2g-1 either the elevated minimal-degree curve or
                      the minimum-energy interior points (minsnap_monomial).
  H  [Rax][2g]        reach rows: control points of b^(k)(t) in degree p-k,
                      k = 1..g, j = 0..p-k (Theorem 1 read as per-axis bounds
                      |b^(k)| <= c_k on the hodograph control points).
  C  [g][p][2g]       cost rows: for d = 0..g-1 the degree-p control points of
                      b^(d)(t) (rows of the state-space matrix P of Eq. (BezDef)),
                      differenced: W_d[l+1] - W_d[l], l = 0..p-1 (Property 2).
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial
from typing import Dict, List

import numpy as np


def _solve_exact(M: List[List[Fraction]], rhs: List[Fraction]) -> List[Fraction]:
    """Gauss-Jordan elimination over the rationals (any non-zero pivot is exact)."""
    n = len(M)
    a = [row[:] + [rhs[i]] for i, row in enumerate(M)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        pv = a[col][col]
        a[col] = [v / pv for v in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col]
                a[r] = [vr - f * vc for vr, vc in zip(a[r], a[col])]
    return [a[r][n] for r in range(n)]


def hermite_monomial(gamma: int, T: Fraction) -> List[List[Fraction]]:
    """Monomial coefficients (in u = t/T) of the minimal-degree Hermite curve.

    Returns a[s][c], s = 0..q, c = 0..2g-1, such that a_s = sum_c a[s][c] xi_c.
    Conditions (Lemma 1): d^c b/dt^c at t=0 equals xL_c and at t=T equals xR_c,
    where d^c/dt^c (u^s) = T^{-c} s!/(s-c)! u^{s-c}.
    """
    g = gamma
    q = 2 * g - 1
    M: List[List[Fraction]] = []
    for c in range(g):  # start conditions
        M.append([Fraction(factorial(s), factorial(s - c)) / T ** c if (s == c) else Fraction(0)
                  for s in range(q + 1)])
    for c in range(g):  # end conditions (u = 1)
        M.append([Fraction(factorial(s), factorial(s - c)) / T ** c if s >= c else Fraction(0)
                  for s in range(q + 1)])
    cols = []
    for c in range(2 * g):
        rhs = [Fraction(1) if r == c else Fraction(0) for r in range(2 * g)]
        cols.append(_solve_exact(M, rhs))
    return [[cols[c][s] for c in range(2 * g)] for s in range(q + 1)]


def minsnap_monomial(gamma: int, p: int, T: Fraction) -> List[List[Fraction]]:
    """Monomial coefficients (in u = t/T) of the degree-p curve meeting the
    Lemma 1 end conditions with minimal energy int_0^T |b^(g+1)(t)|^2 dt.

    Route (independent of the Bernstein normal equations a GPU table generator
    would use): Lagrange conditions of the equality-constrained quadratic
    programme in the p+1 monomial coefficients,
        [2Q  M^T] [a ]   [0  ]
        [M   0  ] [mu] = [rhs],
    with Q_st = int_0^1 s!/(s-g-1)! t!/(t-g-1)! u^(s+t-2g-2) du (the factor
    T^(1-2(g+1)) is a positive constant and does not move the minimiser) and M
    the 2g end conditions of hermite_monomial, solved exactly per column.
    """
    g = gamma
    ne = 2 * g
    nv = p + 1

    def dfac(s):
        return Fraction(factorial(s), factorial(s - g - 1)) if s >= g + 1 else Fraction(0)

    Q = [[(dfac(s) * dfac(t) / (s + t - 2 * g - 1)) if (s >= g + 1 and t >= g + 1) else Fraction(0)
          for t in range(nv)] for s in range(nv)]
    M = []
    for c in range(g):
        M.append([Fraction(factorial(s), factorial(s - c)) / T ** c if s == c else Fraction(0) for s in range(nv)])
    for c in range(g):
        M.append([Fraction(factorial(s), factorial(s - c)) / T ** c if s >= c else Fraction(0) for s in range(nv)])
    K = [[2 * Q[r][c] for c in range(nv)] + [M[e][r] for e in range(ne)] for r in range(nv)]
    K += [[M[e][c] for c in range(nv)] + [Fraction(0)] * ne for e in range(ne)]
    cols = []
    for c in range(ne):
        rhs = [Fraction(0)] * nv + [Fraction(1) if e == c else Fraction(0) for e in range(ne)]
        cols.append(_solve_exact(K, rhs)[:nv])
    return [[cols[c][s] for c in range(ne)] for s in range(nv)]


def derivative_monomial(a: List[List[Fraction]], k: int, T: Fraction) -> List[List[Fraction]]:
    """Monomial coefficients of d^k b/dt^k: a'_r = T^{-k} (r+k)!/r! a_{r+k}."""
    deg = len(a) - 1
    if k > deg:
        return [[Fraction(0)] * len(a[0])]
    return [[a[r + k][c] * Fraction(factorial(r + k), factorial(r)) / T ** k for c in range(len(a[0]))]
            for r in range(deg - k + 1)]


def monomial_to_bernstein(a: List[List[Fraction]], P: int) -> List[List[Fraction]]:
    """beta_l = sum_{s<=l} C(l,s)/C(P,s) a_s, l = 0..P (requires deg a <= P)."""
    deg = len(a) - 1
    assert deg <= P
    ncol = len(a[0])
    out = []
    for l in range(P + 1):
        row = [Fraction(0)] * ncol
        for s in range(min(l, deg) + 1):
            w = Fraction(comb(l, s), comb(P, s))
            for c in range(ncol):
                row[c] += w * a[s][c]
        out.append(row)
    return out


def exact_tables(gamma: int, p: int, T: float, interior: str = "elevate") -> Dict[str, List]:
    """Exact (Fraction) tables for one duration T (T is taken as its exact binary value).

    interior = "elevate": the minimal-degree Hermite curve in degree p (Lemma 1
    plus degree elevation); "minsnap": the degree-p curve with the same end
    conditions and minimal int |b^(g+1)|^2 (equal to "elevate" at p = 2g-1).
    """
    assert p >= 2 * gamma - 1
    Tq = Fraction(T)
    if interior == "minsnap" and p > 2 * gamma - 1:
        a = minsnap_monomial(gamma, p, Tq)
    else:
        a = hermite_monomial(gamma, Tq)
    D = monomial_to_bernstein(a, p)
    H: List[List[Fraction]] = []
    for k in range(1, gamma + 1):
        H.extend(monomial_to_bernstein(derivative_monomial(a, k, Tq), p - k))
    C: List[List[List[Fraction]]] = []
    for d in range(gamma):
        W = monomial_to_bernstein(derivative_monomial(a, d, Tq), p) if d else D
        C.append([[W[l + 1][c] - W[l][c] for c in range(2 * gamma)] for l in range(p)])
    return {"D": D, "H": H, "C": C}


def _to_float(x):
    if isinstance(x, list):
        return [_to_float(v) for v in x]
    return float(x)   # Fraction -> double: correctly rounded (int true division)


def tables(gamma: int, p: int, Ts, interior: str = "elevate") -> Dict[str, np.ndarray]:
    """Double tables for all durations: D [nT][p+1][2g], H [nT][Rax][2g], C [nT][g][p][2g]."""
    Ds, Hs, Cs = [], [], []
    for T in Ts:
        t = exact_tables(gamma, p, float(T), interior)
        Ds.append(_to_float(t["D"]))
        Hs.append(_to_float(t["H"]))
        Cs.append(_to_float(t["C"]))
    return {"D": np.ascontiguousarray(np.array(Ds, dtype=np.float64)),
            "H": np.ascontiguousarray(np.array(Hs, dtype=np.float64)),
            "C": np.ascontiguousarray(np.array(Cs, dtype=np.float64))}


def reach_row_orders(gamma: int, p: int) -> np.ndarray:
    """Derivative order k (1..g) of each reach row, in table order."""
    return np.concatenate([np.full(p - k + 1, k, dtype=np.int32) for k in range(1, gamma + 1)])
