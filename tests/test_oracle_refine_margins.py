"""Pins for the barrier part of the refinement oracle (reach and free margins).

The oracle builds the reach margins of a segment from forward differences of
its control points scaled by p!/(p-k)! T^-k (Theorem 1 read per axis) and the
free margins from the interior control points (Property 1).  Here every
margin is reached by another route:

* reach rows: the segment is expanded into the power basis of u = t/T,
  differentiated k times with numpy, divided by T^k (the chain rule for the
  t-derivative), and converted back to the Bernstein basis of degree p - k by
  the textbook basis change b_j = sum_{i<=j} C(j,i)/C(p-k,i) a_i.  Those are
  the control points of b^(k)(t); the convex-hull property makes them the
  rows Theorem 1 bounds by +-c_k.  The conversion is itself checked against
  direct samples of b^(k)(t).
* free rows: b_r - sum_a A_ra P_la by plain loops over l = 1..p-1 and the
  polytope's rows.

The relaxed log-barrier is restated from its definition, and the oracle's
loss with the snap weight at 0 must equal the sum of the barrier over these
margins.  The gradient of that sum with respect to the control points goes
through the same independent linear maps (applied to unit vectors), and the
duration derivative is a central difference of the independent loss.
Planted mistakes in the oracle's source (a wrong power of T, a shifted bound
index, the end point among the free rows, a sign slip in the free rows) must
each fail.
"""
from __future__ import annotations

import inspect
import types
from math import comb

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from oracle import refine as R
from paper_2411_13507_gb300 import synth
from pins import bernstein_to_power, eval_bernstein, t_derivative_at


def power_to_bernstein(a: np.ndarray) -> np.ndarray:
    """Bernstein coefficients of degree n of the polynomial sum_i a_i u^i (n = len(a) - 1)."""
    n = a.shape[0] - 1
    out = np.zeros(n + 1)
    for j in range(n + 1):
        for i in range(j + 1):
            out[j] += comb(j, i) / comb(n, i) * a[i]
    return out


def hodograph_points(P1: np.ndarray, T: float, k: int) -> np.ndarray:
    """Control points (degree p - k) of d^k b / dt^k for one axis, by the power-basis route."""
    a = bernstein_to_power(np.asarray(P1, dtype=np.float64))
    d = npoly.polyder(a, k) / T ** k
    return power_to_bernstein(d)


def relaxed_barrier(m: float, delta: float) -> float:
    """-log m above delta; below it the quadratic that matches value, slope and curvature at delta."""
    if m >= delta:
        return -np.log(m)
    return -np.log(delta) + 0.5 * ((m - 2.0 * delta) / delta) ** 2 - 0.5


def relaxed_barrier_slope(m: float, delta: float) -> float:
    return -1.0 / m if m >= delta else (m - 2.0 * delta) / delta ** 2


def margins(P: np.ndarray, T: float, A: np.ndarray, b: np.ndarray, nrows: int, bounds):
    """Every margin of one segment with its gradient in the control points: list of (value, d value / d P)."""
    p1, m = P.shape
    p = p1 - 1
    out = []
    for k in range(1, len(bounds) + 1):
        # the linear map P[:, a] -> hodograph control points, column by column
        M = np.stack([hodograph_points(np.eye(p1)[l], T, k) for l in range(p1)], axis=1)
        for a in range(m):
            Q = hodograph_points(P[:, a], T, k)
            assert np.allclose(Q, M @ P[:, a], rtol=1e-12, atol=1e-12 * (1 + np.abs(Q).max()))
            for j in range(p - k + 1):
                for sgn in (-1.0, 1.0):
                    g = np.zeros_like(P)
                    g[:, a] = sgn * M[j]
                    out.append((bounds[k - 1] + sgn * Q[j], g))
    for l in range(1, p):
        for r in range(nrows):
            s = 0.0
            for a in range(m):
                s += A[r, a] * P[l, a]
            g = np.zeros_like(P)
            g[l, :] = -A[r, :m]
            out.append((b[r] - s, g))
    return out


def barrier_loss(P, T, A, b, nrows, bounds, delta):
    return sum(relaxed_barrier(v, delta) for v, _ in margins(P, T, A, b, nrows, bounds))


def barrier_grad(P, T, A, b, nrows, bounds, delta):
    g = np.zeros_like(P)
    for v, dv in margins(P, T, A, b, nrows, bounds):
        g += relaxed_barrier_slope(v, delta) * dv
    return g


@pytest.fixture(scope="module")
def segs():
    rb = synth.refine_segments(seed=11, S=24)
    return rb


def test_hodograph_route_matches_curve_samples(segs):
    """The power-basis route gives the control points of b^(k)(t): their Bezier curve equals sampled derivatives."""
    u = np.linspace(0.0, 1.0, 33)
    for s in range(0, 24, 5):
        for k in (1, 2, 3):
            for a in range(3):
                Q = hodograph_points(segs.P[s, :, a], segs.T[s], k)
                ref = t_derivative_at(segs.P[s, :, a], segs.T[s], k, u)
                assert np.max(np.abs(eval_bernstein(Q, u) - ref)) <= 1e-11 * (1 + np.abs(ref).max())


def test_margins_reach_both_barrier_branches(segs):
    """The fixture exercises the log branch and the quadratic branch for reach and free rows."""
    d = 0.1
    reach_lo = reach_hi = free_lo = free_hi = 0
    for s in range(24):
        ms = margins(segs.P[s], segs.T[s], segs.A[s], segs.b[s], int(segs.nrows[s]), segs.bounds)
        nreach = sum(3 * (8 - k) * 2 for k in (1, 2, 3))
        for i, (v, _) in enumerate(ms):
            if i < nreach:
                reach_lo += v < d
                reach_hi += v >= d
            else:
                free_lo += v < d
                free_hi += v >= d
    assert min(reach_lo, reach_hi, free_hi) > 0


@pytest.mark.parametrize("delta", [0.1, 2.0])
def test_barrier_loss_equals_independent_margins(segs, delta):
    loss, dP, dT = R.loss_and_grad(segs.P, segs.T, segs.A, segs.b, segs.nrows, segs.bounds,
                                   w_snap=0.0, mu=1.0, delta=delta)
    for s in range(24):
        args = (segs.P[s], segs.T[s], segs.A[s], segs.b[s], int(segs.nrows[s]), segs.bounds)
        ref = barrier_loss(*args, delta)
        assert abs(loss[s] - ref) <= 1e-12 * max(1.0, abs(ref)), (s, loss[s], ref)
        gref = barrier_grad(*args, delta)
        assert np.max(np.abs(dP[s] - gref)) <= 1e-10 * max(1.0, np.abs(gref).max()), s
        h = 1e-6 * segs.T[s]
        fp = barrier_loss(segs.P[s], segs.T[s] + h, *args[2:], delta)
        fm = barrier_loss(segs.P[s], segs.T[s] - h, *args[2:], delta)
        fd = (fp - fm) / (2 * h)
        assert abs(dT[s] - fd) <= 1e-6 * max(1.0, abs(fd)), (s, dT[s], fd)


def test_barrier_with_free_rows_in_quadratic_branch(segs):
    """Tighten every polytope so some interior control points sit closer than delta (or outside)."""
    b = segs.b.copy()
    valid = np.arange(segs.A.shape[1])[None, :] < segs.nrows[:, None]
    inner = np.einsum("sra,sla->slr", segs.A, segs.P[:, 1:7, :]).max(axis=1)
    b = np.where(valid, inner + np.linspace(-0.3, 0.05, b.shape[1])[None, :], b)
    loss, dP, _ = R.loss_and_grad(segs.P, segs.T, segs.A, b, segs.nrows, segs.bounds, w_snap=0.0, mu=1.0, delta=0.1)
    lows = 0
    for s in range(24):
        args = (segs.P[s], segs.T[s], segs.A[s], b[s], int(segs.nrows[s]), segs.bounds)
        lows += sum(v < 0.1 for v, _ in margins(*args)[-(6 * int(segs.nrows[s])):])
        ref = barrier_loss(*args, 0.1)
        assert abs(loss[s] - ref) <= 1e-12 * max(1.0, abs(ref))
        assert np.max(np.abs(dP[s] - barrier_grad(*args, 0.1))) <= 1e-10 * max(1.0, np.abs(dP[s]).max())
    assert lows > 0


MISTAKES = {
    "power of T one short": ("T[:, None, None] ** (-k)", "T[:, None, None] ** (-(k - 1))"),
    "bound of the next order": ("bounds[k - 1] + sign * Q", "bounds[k % gamma] + sign * Q"),
    "end point among the free rows": ("for l in range(1, p):", "for l in range(1, p + 1):"),
    "sign slip in the free rows": ('mg = b - np.einsum("sra,sa->sr"', 'mg = b + np.einsum("sra,sa->sr"'),
}


def planted(old: str, new: str) -> types.ModuleType:
    src = inspect.getsource(R)
    assert src.count(old) == 1, old
    mod = types.ModuleType("refine_planted")
    exec(compile(src.replace(old, new), "refine_planted", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_margin_mistakes_are_caught(segs, name):
    bad = planted(*MISTAKES[name])
    loss, _, _ = bad.loss_and_grad(segs.P, segs.T, segs.A, segs.b, segs.nrows, segs.bounds, w_snap=0.0, mu=1.0)
    worst = 0.0
    for s in range(24):
        ref = barrier_loss(segs.P[s], segs.T[s], segs.A[s], segs.b[s], int(segs.nrows[s]), segs.bounds, 0.1)
        worst = max(worst, abs(loss[s] - ref) / max(1.0, abs(ref)))
    assert worst > 1e-6, name
