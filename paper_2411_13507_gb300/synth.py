"""Seeded synthetic planning workloads (inputs only).

This module draws the inputs that both the CUDA path and the CPU oracle
consume: sampled reduced-order states, convex free-space polytopes in
H-representation (A x <= b), the candidate durations T and start/goal
positions.  It holds none of the planner's arithmetic -- no control points,
no reachable-polytope rows, no costs, no membership decisions -- it only
samples numbers.  Every draw comes from a counter-based SplitMix64 stream, so
each array is a pure function of (recipe, seed) on every platform and numpy
version.

Recipes (sizes follow the workloads the method is evaluated on):

* ``double_integrator_2d``  -- 2-D double integrator (|v| <= 2, |a| <= 4),
  domain [0,10]^2, 16 polytopes of 4-8 rows, 512 states, degree 5,
  8 durations in [0.2, 2], FP64.
* ``triple_integrator_3d``  -- 3-D triple integrator (|v| <= 3, |a| <= 6,
  |jerk| <= 30), domain [0,20]^3, 64 polytopes of 6-12 rows, 8192 states,
  degree 7, 16 durations log-uniform in [0.1, 3], FP32-representable values.
* ``batched_queries``       -- many independent triple-integrator queries of
  uneven size (states log-uniform in [512, 16384], polytopes 8-128,
  durations 8-16).
* ``refine_segments``       -- degree-7 3-D segments for the smoothed-barrier
  refinement (interior control points N(0,1) around a straight line).
* ``mpc_references``        -- reference nodes for the MPC refinement: each a
  cubic polynomial in time per axis (random start inside the box, speed
  U[0.2, 1], acceleration and jerk N(0, 0.5)) sampled at k dt with its
  derivatives up to gamma - 1, kept when every sample stays in the inner 90%
  of the box.

Polytope recipe: an axis box (centre uniform in the domain, side uniform in
[smin, smax] per axis) intersected with 0..max_cuts random half-spaces whose
unit normal is uniform on the sphere and whose offset is
n.c + U[0.2, 0.9] * (sum_a |n_a| h_a), so the box centre stays interior.
States: a polytope chosen uniformly, a position uniform in it (rejection from
its box), every higher derivative uniform in [-1, 1] per axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter-based SplitMix64 stream: output k is mix(s0 + k * golden)."""

    def __init__(self, seed: int, tag: int = 0):
        base = np.array([(int(seed) * 0x9E3779B97F4A7C15 + int(tag) * 0xD1B54A32D192ED03) & _MASK],
                        dtype=np.uint64)
        self._s0 = _mix64(base)[0]
        self._n = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self._n + 1, self._n + n + 1, dtype=np.uint64)
        self._n += n
        with np.errstate(over="ignore"):
            return _mix64(self._s0 + k * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        return lo + (self.u64(n) % np.uint64(span)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        u1 = np.where(u1 <= 0.0, 2.0 ** -53, u1)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Model:
    """Chain-of-integrators planning model: m outputs, relative degree gamma.

    ``bounds[k-1]`` is the per-axis bound on the k-th derivative, k = 1..gamma
    (k = gamma is the input).  ``degree`` is the Bezier degree p >= 2*gamma-1.
    """
    m: int
    gamma: int
    degree: int
    bounds: Sequence[float]
    tighten: float = 0.0
    cost_mode: str = "state"   # "state": all n rows of the state-space control points; "pos": position only
    interior: str = "elevate"  # interior control points for degree > 2*gamma-1: "elevate" or "minsnap"

    @property
    def n(self) -> int:
        return self.m * self.gamma


@dataclass
class Problem:
    """One planning query: states [N][n] stacked [pos; vel; acc...] per state."""
    name: str
    seed: int
    model: Model
    dtype: str                      # "f64" or "f32": values are representable in this type
    states: np.ndarray              # float64 [N][n]
    T: np.ndarray                   # float64 [nT], ascending
    poly_off: np.ndarray            # int32 [K+1]
    A: np.ndarray                   # float64 [R][m]
    b: np.ndarray                   # float64 [R]
    start_pos: np.ndarray           # float64 [m]
    goal_pos: np.ndarray            # float64 [m]
    domain: tuple = field(default=(0.0, 1.0))

    @property
    def N(self) -> int:
        return int(self.states.shape[0])

    @property
    def K(self) -> int:
        return int(self.poly_off.shape[0] - 1)

    @property
    def nT(self) -> int:
        return int(self.T.shape[0])


def _round(x: np.ndarray, dtype: str) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    if dtype == "f32":
        return x.astype(np.float32).astype(np.float64)
    return x


def _polytopes(rng: SplitMix64, m: int, K: int, domain, side, max_cuts, dtype):
    lo, hi = domain
    centers = rng.uniform(K * m, lo, hi).reshape(K, m)
    halves = 0.5 * rng.uniform(K * m, side[0], side[1]).reshape(K, m)
    ncuts = rng.integers(K, 0, max_cuts)
    rows_A: List[np.ndarray] = []
    rows_b: List[float] = []
    off = [0]
    boxes = []
    for k in range(K):
        c, h = centers[k], halves[k]
        for a in range(m):
            e = np.zeros(m)
            e[a] = 1.0
            rows_A.append(e.copy())
            rows_b.append(c[a] + h[a])
            rows_A.append(-e)
            rows_b.append(-(c[a] - h[a]))
        for _ in range(int(ncuts[k])):
            nrm = rng.normal(m)
            nn = float(np.sqrt(np.sum(nrm * nrm)))
            if nn == 0.0:
                nrm = np.ones(m)
                nn = float(np.sqrt(m))
            nrm = nrm / nn
            frac = rng.uniform(1, 0.2, 0.9)[0]
            rows_A.append(nrm)
            rows_b.append(float(nrm @ c) + frac * float(np.abs(nrm) @ h))
        off.append(len(rows_b))
        boxes.append((c - h, c + h))
    A = _round(np.array(rows_A, dtype=np.float64).reshape(-1, m), dtype)
    b = _round(np.array(rows_b, dtype=np.float64), dtype)
    return np.array(off, dtype=np.int32), A, b, boxes


def _inside(A, b, lo_row, hi_row, x):
    """Sampling acceptance: x strictly inside rows [lo_row, hi_row) (margin 1e-9)."""
    s = A[lo_row:hi_row] @ x
    return bool(np.all(s <= b[lo_row:hi_row] - 1e-9))


def _sample_in_polytopes(rng, which, poly_off, A, b, boxes, m, dtype):
    """Uniform points in the chosen polytopes, by rejection from each box."""
    n = len(which)
    out = np.zeros((n, m))
    pending = np.arange(n)
    for _ in range(10000):
        if pending.size == 0:
            break
        u = rng.uniform(pending.size * m).reshape(pending.size, m)
        keep = []
        for idx, row in zip(pending, u):
            k = int(which[idx])
            lo, hi = boxes[k]
            x = _round(lo + (hi - lo) * row, dtype)
            if _inside(A, b, poly_off[k], poly_off[k + 1], x):
                out[idx] = x
            else:
                keep.append(idx)
        pending = np.array(keep, dtype=np.int64)
    if pending.size:
        raise RuntimeError("rejection sampling did not converge")
    return out


def make_problem(name: str, seed: int, model: Model, N: int, K: int, T: np.ndarray,
                 domain=(0.0, 10.0), side=(2.0, 5.0), max_cuts=4, dtype="f64") -> Problem:
    rng_poly = SplitMix64(seed, 1)
    rng_state = SplitMix64(seed, 2)
    rng_query = SplitMix64(seed, 3)
    m, g = model.m, model.gamma
    poly_off, A, b, boxes = _polytopes(rng_poly, m, K, domain, side, max_cuts, dtype)
    which = rng_state.integers(N, 0, K - 1) if K > 0 else np.zeros(N, dtype=np.int64)
    states = np.zeros((N, model.n))
    if N and K:
        states[:, :m] = _sample_in_polytopes(rng_state, which, poly_off, A, b, boxes, m, dtype)
    elif N:
        states[:, :m] = rng_state.uniform(N * m, domain[0], domain[1]).reshape(N, m)
    for c in range(1, g):
        states[:, c * m:(c + 1) * m] = rng_state.uniform(N * m, -1.0, 1.0).reshape(N, m)
    states = _round(states, dtype)
    if K >= 2:
        ks = rng_query.integers(1, 0, K - 1)[0]
        kg = (ks + 1 + rng_query.integers(1, 0, K - 2)[0]) % K
    else:
        ks = kg = 0
    if K:
        sg = _sample_in_polytopes(rng_query, np.array([ks, kg]), poly_off, A, b, boxes, m, dtype)
    else:
        sg = rng_query.uniform(2 * m, domain[0], domain[1]).reshape(2, m)
    return Problem(name=name, seed=seed, model=model, dtype=dtype, states=states,
                   T=_round(np.asarray(T, dtype=np.float64), dtype), poly_off=poly_off, A=A, b=b,
                   start_pos=_round(sg[0], dtype), goal_pos=_round(sg[1], dtype), domain=domain)


@dataclass
class Obstacles:
    """Convex obstacle polytopes {z : A z <= b} in position space (CSR rows)."""
    off: np.ndarray                 # int32 [n+1]
    A: np.ndarray                   # float64 [R][m]
    b: np.ndarray                   # float64 [R]

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)


def obstacles(seed: int, n: int, m: int, domain=(0.0, 20.0), side=(0.3, 1.2), max_cuts: int = 3,
              dtype: str = "f64") -> Obstacles:
    """n random convex obstacles: axis boxes (centre U(domain), side U(side))
    cut by 0..max_cuts random planes, as for the free polytopes."""
    off, A, b, _ = _polytopes(SplitMix64(seed, 4), m, n, domain, side, max_cuts, dtype)
    return Obstacles(off, A, b)


def keepout_2d(seed: int = 1, N: int = 5000, n_obst: int = 500, T: float = 0.5, width: float = 5.0,
               dtype: str = "f64"):
    """The keep-out setting of the paper's experiments: 2-D double integrator
    (|v| <= 2, |a| <= 4, degree 5), one free box [0, width]^2, N states with
    uniform positions and velocities U[-1, 1], curves of one duration T (the
    defaults give about 5000 nodes and 46,000 edges, the scale of the paper's
    maze and random-obstacle runs), and n_obst random convex obstacles (boxes
    with sides U[0.005, 0.02] * width cut by up to 3 planes; at the defaults
    they remove about 40% of the edges).  Returns (problem, obstacles)."""
    model = Model(2, 2, 5, (2.0, 4.0))
    rng = SplitMix64(seed, 2)
    states = np.zeros((N, 4))
    states[:, :2] = rng.uniform(N * 2, 0.0, width).reshape(N, 2)
    states[:, 2:] = rng.uniform(N * 2, -1.0, 1.0).reshape(N, 2)
    A = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])
    b = np.array([width, 0.0, width, 0.0])
    rq = SplitMix64(seed, 3)
    sg = rq.uniform(4, 0.05 * width, 0.95 * width).reshape(2, 2)
    prob = Problem(name="keepout_2d", seed=seed, model=model, dtype=dtype, states=_round(states, dtype),
                   T=_round(np.array([T], dtype=np.float64), dtype), poly_off=np.array([0, 4], dtype=np.int32),
                   A=A, b=b, start_pos=_round(sg[0], dtype), goal_pos=_round(sg[1], dtype), domain=(0.0, width))
    return prob, obstacles(seed, n_obst, 2, (0.0, width), (0.005 * width, 0.02 * width), 3, dtype)


def double_integrator_2d(seed: int = 1, N: int = 512, K: int = 16, nT: int = 8,
                         degree: int = 5, dtype: str = "f64") -> Problem:
    """2-D double integrator, |v| <= 2, |a| <= 4, domain [0,10]^2, 4-8 rows per polytope."""
    model = Model(m=2, gamma=2, degree=degree, bounds=(2.0, 4.0))
    T = np.linspace(0.2, 2.0, nT)
    return make_problem("double_integrator_2d", seed, model, N, K, T, domain=(0.0, 10.0),
                        side=(2.0, 5.0), max_cuts=4, dtype=dtype)


def _log_uniform_T(seed: int, nT: int, lo=0.1, hi=3.0) -> np.ndarray:
    r = SplitMix64(seed, 4)
    return np.sort(np.exp(r.uniform(nT, np.log(lo), np.log(hi))))


def triple_integrator_3d(seed: int = 1, N: int = 8192, K: int = 64, nT: int = 16,
                         degree: int = 7, dtype: str = "f32") -> Problem:
    """3-D triple integrator, |v| <= 3, |a| <= 6, |jerk| <= 30, domain [0,20]^3, 6-12 rows."""
    model = Model(m=3, gamma=3, degree=degree, bounds=(3.0, 6.0, 30.0))
    T = _log_uniform_T(seed, nT)
    return make_problem("triple_integrator_3d", seed, model, N, K, T, domain=(0.0, 20.0),
                        side=(2.0, 6.0), max_cuts=6, dtype=dtype)


def batched_queries(seed: int = 1, Q: int = 256, n_lo: int = 512, n_hi: int = 16384,
                    k_lo: int = 8, k_hi: int = 128, t_lo: int = 8, t_hi: int = 16) -> List[Problem]:
    """Many independent triple-integrator queries of uneven size (one seed each)."""
    r = SplitMix64(seed, 5)
    Ns = np.floor(np.exp(r.uniform(Q, np.log(n_lo), np.log(n_hi + 1)))).astype(np.int64)
    Ns = np.clip(Ns, n_lo, n_hi)
    Ks = r.integers(Q, k_lo, k_hi)
    nTs = r.integers(Q, t_lo, t_hi)
    out = []
    for q in range(Q):
        qseed = int(seed) * 100003 + q
        out.append(triple_integrator_3d(seed=qseed, N=int(Ns[q]), K=int(Ks[q]), nT=int(nTs[q])))
    return out


@dataclass
class RefineBatch:
    """Degree-p segments with one free-space polytope each (rows padded to rmax)."""
    P: np.ndarray          # float64 [S][p+1][m]
    T: np.ndarray          # float64 [S]
    A: np.ndarray          # float64 [S][rmax][m]  (padded rows are zero with b = 1)
    b: np.ndarray          # float64 [S][rmax]
    nrows: np.ndarray      # int32 [S]
    bounds: Sequence[float]


def refine_segments(seed: int = 1, S: int = 65536, degree: int = 7, m: int = 3,
                    rmax: int = 12, max_cuts: int = 6, bounds=(3.0, 6.0, 30.0)) -> RefineBatch:
    """Segments: end points on a random line, interior points = line points + N(0,1).

    The free polytope of a segment is the bounding box of its control points
    inflated by U[1,3] per axis, cut by random half-spaces that keep the whole
    control polygon inside (the offset is the largest n.P_l plus U[0.1, 1]).
    T ~ U[0.2, 2].
    """
    r = SplitMix64(seed, 6)
    p = degree
    p0 = r.uniform(S * m, 0.0, 20.0).reshape(S, m)
    d = r.normal(S * m).reshape(S, m)
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-12)
    L = r.uniform(S, 1.0, 4.0)[:, None]
    P = np.zeros((S, p + 1, m))
    for l in range(p + 1):
        P[:, l, :] = p0 + (l / p) * L * d
    P[:, 1:p, :] += r.normal(S * (p - 1) * m).reshape(S, p - 1, m)
    T = r.uniform(S, 0.2, 2.0)
    A = np.zeros((S, rmax, m))
    b = np.ones((S, rmax))
    nrows = np.zeros(S, dtype=np.int32)
    lo = P.min(axis=1) - r.uniform(S * m, 1.0, 3.0).reshape(S, m)
    hi = P.max(axis=1) + r.uniform(S * m, 1.0, 3.0).reshape(S, m)
    ncut = r.integers(S, 0, max_cuts)
    nrm = r.normal(S * max_cuts * m).reshape(S, max_cuts, m)
    nrm /= np.maximum(np.linalg.norm(nrm, axis=2, keepdims=True), 1e-12)
    slack = r.uniform(S * max_cuts, 0.1, 1.0).reshape(S, max_cuts)
    for s in range(S):
        rows = 0
        for a in range(m):
            A[s, rows, a] = 1.0
            b[s, rows] = hi[s, a]
            rows += 1
            A[s, rows, a] = -1.0
            b[s, rows] = -lo[s, a]
            rows += 1
        for c in range(int(ncut[s])):
            if rows >= rmax:
                break
            A[s, rows] = nrm[s, c]
            b[s, rows] = float(np.max(P[s] @ nrm[s, c])) + slack[s, c]
            rows += 1
        nrows[s] = rows
    return RefineBatch(P=P, T=T, A=A, b=b, nrows=nrows, bounds=tuple(bounds))


def mpc_references(seed: int, B: int, H: int, dt: float, width: float = 5.0, m: int = 2, g: int = 2) -> np.ndarray:
    """[B][H+1][m g] reference nodes (derivative-major: positions, then
    velocities, ...): samples of cubic polynomials in time and their
    derivatives (the recipe above)."""
    rng = SplitMix64(seed, 11)
    out = np.zeros((B, H + 1, m * g))
    t = dt * np.arange(H + 1)
    b = 0
    while b < B:
        p0 = rng.uniform(m, 0.1 * width, 0.9 * width)
        d = rng.normal(m)
        d = d / max(float(np.linalg.norm(d)), 1e-12)
        v0 = d * float(rng.uniform(1, 0.2, 1.0)[0])
        a0 = 0.5 * rng.normal(m)
        j0 = 0.5 * rng.normal(m)
        # derivative c of p0 + v0 t + a0 t^2 / 2 + j0 t^3 / 6
        coef = [p0, v0, a0, j0]
        nodes = np.zeros((H + 1, m * g))
        for c in range(g):
            val = np.zeros((H + 1, m))
            for e in range(c, 4):
                fac = 1.0
                for q in range(e - c + 1, e + 1):
                    fac *= q
                val += np.outer(t ** (e - c), coef[e]) * (fac / np.prod(np.arange(1, e + 1), dtype=np.float64))
            nodes[:, c * m:(c + 1) * m] = val
        pos = nodes[:, :m]
        if np.all(pos >= 0.05 * width) and np.all(pos <= 0.95 * width):
            out[b] = nodes
            b += 1
    return out
