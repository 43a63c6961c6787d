"""Pins for the keep-out cut oracle (oracle/cut.py; Sec. III-B, Algorithm 2,
Cut-QP).  Expected values come from brute force on tiny games, from
straight-segment geometry with the slab method, from random points of the
hull, and from the optimality certificates of the exact matrix-game solution.
"""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import oracle
from oracle import cut as OC
from paper_2411_13507_gb300 import synth


def brute_two_row_game(G):
    """min over lambda in [0,1] of max_r (lambda G[0,r] + (1-lambda) G[1,r]),
    exactly: the optimum is at an end point or where two column lines cross."""
    a = [Fraction(float(v)) for v in G[0]]
    b = [Fraction(float(v)) for v in G[1]]
    cands = {Fraction(0), Fraction(1)}
    for r, s in combinations(range(len(a)), 2):
        den = (a[r] - b[r]) - (a[s] - b[s])
        if den != 0:
            lam = (b[s] - b[r]) / den
            if 0 <= lam <= 1:
                cands.add(lam)
    return min(max(lam * a[r] + (1 - lam) * b[r] for r in range(len(a))) for lam in cands)


@pytest.mark.parametrize("seed", range(12))
def test_game_value_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(2, int(rng.integers(1, 6)))).round(3)
    v, lam, y = OC.game_value(G)
    assert v == brute_two_row_game(G)


@pytest.mark.parametrize("seed", range(8))
def test_game_value_duality_certificate(seed):
    """lambda and y from the simplex certify optimality: max_r (G^T lambda)_r
    equals min_l (G y)_l equals the value, with both on their simplices."""
    rng = np.random.default_rng(100 + seed)
    G = rng.normal(size=(int(rng.integers(2, 9)), int(rng.integers(2, 10))))
    v, lam, y = OC.game_value(G)
    Gf = [[Fraction(float(x)) for x in row] for row in G]
    assert all(x >= 0 for x in lam) and sum(lam) == 1
    assert all(x >= 0 for x in y) and sum(y) == 1
    upper = max(sum(lam[l] * Gf[l][r] for l in range(len(lam))) for r in range(len(y)))
    lower = min(sum(y[r] * Gf[l][r] for r in range(len(y))) for l in range(len(lam)))
    assert upper == v == lower


def test_textbook_games():
    # matching pennies (value 0); a dominated row; a saddle point
    assert OC.game_value(np.array([[1.0, -1.0], [-1.0, 1.0]]))[0] == 0
    assert OC.game_value(np.array([[3.0, 2.0], [1.0, 0.5]]))[0] == Fraction(1)
    assert OC.game_value(np.array([[2.0, 4.0], [3.0, 1.0]]))[0] == Fraction(5, 2)


def slab_hit(p0, p1, lo, hi):
    """Closed segment [p0, p1] meets the closed box [lo, hi] (slab method)."""
    t0, t1 = 0.0, 1.0
    for a in range(len(p0)):
        d = p1[a] - p0[a]
        if d == 0.0:
            if p0[a] < lo[a] or p0[a] > hi[a]:
                return False, 0.0
            continue
        ta, tb = (lo[a] - p0[a]) / d, (hi[a] - p0[a]) / d
        if ta > tb:
            ta, tb = tb, ta
        t0, t1 = max(t0, ta), min(t1, tb)
    return t0 <= t1, t1 - t0


def rest_problem(seed, N=48, n_obst=24, width=4.0):
    """States at rest: every curve is the straight segment between positions."""
    prob, _ = synth.keepout_2d(seed, N=N, n_obst=1, width=width)
    prob.states[:, 2:] = 0.0
    prob.model.bounds = (50.0, 500.0)   # every pair reachable
    rng = np.random.default_rng(seed)
    lo = rng.uniform(0.0, width, size=(n_obst, 2))
    hi = lo + rng.uniform(0.1, 0.6, size=(n_obst, 2))
    A = np.tile(np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]), (n_obst, 1))
    b = np.concatenate([[h[0], -l[0], h[1], -l[1]] for l, h in zip(lo, hi)])
    off = np.arange(0, 4 * n_obst + 1, 4)
    return prob, off, A, b, lo, hi


@pytest.mark.parametrize("seed", [1, 2])
def test_cut_equals_slab_method_on_straight_segments(seed):
    prob, off, A, b, lo, hi = rest_problem(seed)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    r = OC.cut(op, csr, off, A, b)
    kept = {(i, int(j)) for i in range(prob.N) for j in r["col"][r["row_off"][i]:r["row_off"][i + 1]]}
    ro = csr["row_off"]
    checked = 0
    for i in range(prob.N):
        for j in csr["col"][ro[i]:ro[i + 1]]:
            p0, p1 = prob.states[i, :2], prob.states[j, :2]
            hits = [slab_hit(p0, p1, lo[o], hi[o]) for o in range(len(lo))]
            if any(h and abs(w) < 1e-9 for h, w in hits):
                continue   # grazing contact: left to rounding
            expect_kept = not any(h for h, _ in hits)
            assert ((i, int(j)) in kept) == expect_kept, (i, j)
            checked += 1
    assert checked > 500 and r["steps"][1] > 0 and r["steps"][2] > 0


@pytest.mark.parametrize("seed", range(3))
def test_hit_decisions_against_hull_samples_and_certificates(seed):
    """Every obstacle decision of a random workload: a hull point sampled
    inside the obstacle forces 'hit'; a 'miss' decided by the matrix game comes
    with a separating hyperplane that clears every control point."""
    prob, obs = synth.keepout_2d(seed + 5, N=300, n_obst=40)
    op = oracle.OracleProblem(prob)
    e = op.edges(with_detail=True)
    rng = np.random.default_rng(seed)
    idx = np.nonzero(e["mask"])[0][:150]
    n_lp = 0
    for k in idx:
        i, j = int(e["i"][k]), int(e["j"][k])
        P = OC.control_points(op.D[0], op.gamma, op.m, op.states[i], op.states[j])
        W = rng.dirichlet(np.ones(P.shape[0]), size=400)
        Z = np.concatenate([W @ P, P])
        for o in range(obs.n):
            A, b = obs.A[obs.off[o]:obs.off[o + 1]], obs.b[obs.off[o]:obs.off[o + 1]]
            G = OC.margins(P, A, b)
            hit, step, v = OC.obstacle_hit(G)
            inside = np.all(Z @ A.T - b <= -1e-12, axis=1)
            if inside.any():
                assert hit
            if step == 3:
                n_lp += 1
                val, lam, y = OC.game_value(G)
                if not hit:
                    h = np.array([float(x) for x in y]) @ A
                    beta = float(np.array([float(x) for x in y]) @ b)
                    assert np.all(P @ h - beta > -1e-12)
                else:
                    z = np.array([float(x) for x in lam]) @ P
                    assert np.all(A @ z - b <= 1e-9)
    assert n_lp > 0


def test_planted_mistakes_are_caught():
    """A sign slip in the margins or skipping the matrix game changes the cut
    of the straight-segment workload."""
    prob, off, A, b, lo, hi = rest_problem(3)
    op = oracle.OracleProblem(prob)
    csr = op.csr(with_detail=True)
    good = OC.cut(op, csr, off, A, b)
    orig_margins, orig_hit = OC.margins, OC.obstacle_hit
    try:
        OC.margins = lambda P, A_, b_: orig_margins(P, A_, -b_)
        bad = OC.cut(op, csr, off, A, b)
        assert not np.array_equal(bad["col"], good["col"])
        OC.margins = orig_margins

        def no_game(G):
            hit, step, v = orig_hit(G)
            return (False, step, v) if step == 3 else (hit, step, v)
        OC.obstacle_hit = no_game
        bad = OC.cut(op, csr, off, A, b)
        assert len(bad["col"]) > len(good["col"])
    finally:
        OC.margins, OC.obstacle_hit = orig_margins, orig_hit
