"""Pins for the oracle's pair test, membership, nearest vertex and Dijkstra.

Expected values come from brute force written from the definitions
(tests/pins.py: control points -> textbook hodograph -> bounds; A P <= b;
state-space polygon length), dense sampling of the curve (Property 1),
numerical arc length (Property 2), symmetry/monotonicity/translation
invariants, and exhaustive path enumeration on tiny graphs.
"""
import itertools
import os
import shutil
import subprocess
from math import factorial

import numpy as np
import pytest

import oracle
from oracle import tables as T_
from paper_2411_13507_gb300 import synth
import pins


def small_problem(seed=3, N=48, K=4, nT=5, gamma=2, degree=5, dtype="f64"):
    if gamma == 2:
        pr = synth.double_integrator_2d(seed=seed, N=N, K=K, nT=nT, degree=degree, dtype=dtype)
    else:
        pr = synth.triple_integrator_3d(seed=seed, N=N, K=K, nT=nT, degree=degree, dtype=dtype)
    return pr


def _xi(op, i, j, a):
    m, g = op.m, op.gamma
    return np.array([op.states[i, c * m + a] for c in range(g)] + [op.states[j, c * m + a] for c in range(g)])


@pytest.mark.parametrize("gamma,degree,dtype", [(2, 5, "f64"), (3, 7, "f32"), (2, 3, "f64"), (3, 5, "f64")])
def test_pairs_match_brute_force(gamma, degree, dtype):
    pr = small_problem(gamma=gamma, degree=degree, dtype=dtype, N=40, K=3, nT=6)
    op = oracle.OracleProblem(pr)
    inm = op.membership()
    e = op.edges()
    assert e["i"].size > 50
    mdl = pr.model
    checked = 0
    for idx in range(e["i"].size):
        i, j = int(e["i"][idx]), int(e["j"][idx])
        shared = np.nonzero(inm[i] & inm[j])[0]
        assert shared.size and i != j
        for t, T in enumerate(pr.T):
            D = op.D[t]
            best_f = -np.inf
            for k in shared:
                lo, hi = pr.poly_off[k], pr.poly_off[k + 1]
                rm, fm, cost = pins.brute_pair(mdl.m, mdl.gamma, mdl.degree, np.asarray(mdl.bounds), T, D,
                                               pr.A[lo:hi], pr.b[lo:hi], pr.states[i], pr.states[j], mdl.cost_mode)
                best_f = max(best_f, fm)
            scale_r = 1.0 + abs(rm)
            assert abs(e["rmarg"][idx, t] - rm) <= 1e-9 * (1 + np.max(np.abs(op.H[t])) * 10), (rm, e["rmarg"][idx, t])
            assert abs(e["fmarg"][idx, t] - best_f) <= 1e-9 * (1 + abs(best_f))
            assert abs(e["costs"][idx, t] - cost) <= 1e-9 * cost
            if abs(rm) > 1e-7 * scale_r and abs(best_f) > 1e-7:
                bit = (rm >= 0) and (best_f >= 0)
                assert bool((e["mask"][idx] >> t) & 1) == bit
                checked += 1
        fe = [t for t in range(pr.nT) if (e["mask"][idx] >> t) & 1]
        if fe:
            tb = min(fe, key=lambda t: (e["costs"][idx, t], t))
            assert e["t"][idx] == tb and e["w"][idx] == e["costs"][idx, tb]
        else:
            assert e["t"][idx] == -1 and np.isinf(e["w"][idx])
    assert checked > 100


def test_candidates_are_exactly_the_sharing_pairs():
    pr = small_problem(N=60, K=5)
    op = oracle.OracleProblem(pr)
    inm = op.membership().astype(bool)
    e = op.edges(with_detail=False)
    got = set(zip(e["i"].tolist(), e["j"].tolist()))
    want = {(i, j) for i in range(pr.N) for j in range(pr.N) if i != j and np.any(inm[i] & inm[j])}
    assert got == want
    # rows sorted by j
    for i in range(pr.N):
        js = e["j"][e["i"] == i]
        assert np.all(np.diff(js) > 0)


def test_membership_brute_force():
    pr = small_problem(N=200, K=8)
    op = oracle.OracleProblem(pr)
    inm = op.membership()
    for k in range(pr.K):
        lo, hi = pr.poly_off[k], pr.poly_off[k + 1]
        s = pr.states[:, :2] @ pr.A[lo:hi].T - pr.b[lo:hi][None, :]
        decided = np.all(np.abs(s) > 1e-12, axis=1)
        want = np.all(s <= 0, axis=1)
        assert np.array_equal(inm[decided, k].astype(bool), want[decided])


def test_hull_invariant_dense_sampling():
    """Property 1: whenever the oracle marks (pair, T) feasible, the sampled curve
    and its derivatives (1025 points) satisfy every bound and stay inside a
    shared polytope.  One-sided (the control-point test is conservative)."""
    for gamma, degree in [(2, 5), (3, 7)]:
        pr = small_problem(gamma=gamma, degree=degree, N=60, K=3, nT=8, seed=11)
        op = oracle.OracleProblem(pr)
        inm = op.membership()
        e = op.edges()
        mdl = pr.model
        u = np.linspace(0.0, 1.0, 1025)
        n_feas = 0
        for idx in np.nonzero(e["mask"])[0][:300]:
            i, j = int(e["i"][idx]), int(e["j"][idx])
            for t in range(pr.nT):
                if not (e["mask"][idx] >> t) & 1:
                    continue
                n_feas += 1
                T = pr.T[t]
                pts = np.stack([pins.eval_bernstein(op.D[t] @ _xi(op, i, j, a), u) for a in range(mdl.m)], axis=1)
                for k in range(1, mdl.gamma + 1):
                    for a in range(mdl.m):
                        dk = pins.t_derivative_at(op.D[t] @ _xi(op, i, j, a), T, k, u)
                        assert np.all(np.abs(dk) <= mdl.bounds[k - 1] + 1e-9)
                ok_any = False
                for k in np.nonzero(inm[i] & inm[j])[0]:
                    lo, hi = pr.poly_off[k], pr.poly_off[k + 1]
                    if np.all(pts @ pr.A[lo:hi].T <= pr.b[lo:hi] + 1e-9):
                        ok_any = True
                assert ok_any
        assert n_feas > 20


def test_time_reversal_symmetry():
    """(i -> j, T) feasible iff (j' -> i', T) feasible where ' negates the odd
    derivatives; the two curves are time reversals, so costs are equal."""
    pr = small_problem(N=50, K=3, nT=6, seed=5)
    rev = synth.double_integrator_2d(seed=5, N=50, K=3, nT=6)
    m, g = pr.model.m, pr.model.gamma
    for c in range(1, g, 2):
        rev.states[:, c * m:(c + 1) * m] *= -1.0
    a = oracle.OracleProblem(pr).edges()
    b = oracle.OracleProblem(rev).edges()
    idx_b = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(b["i"], b["j"]))}
    for k, (i, j) in enumerate(zip(a["i"], a["j"])):
        kb = idx_b[(int(j), int(i))]
        np.testing.assert_allclose(a["costs"][k], b["costs"][kb], rtol=1e-12)
        np.testing.assert_allclose(a["rmarg"][k], b["rmarg"][kb], rtol=1e-9, atol=1e-9)
        close = (np.abs(a["rmarg"][k]) < 1e-9) | (np.abs(a["fmarg"][k]) < 1e-9)
        bits_a = np.array([(a["mask"][k] >> t) & 1 for t in range(pr.nT)])
        bits_b = np.array([(b["mask"][kb] >> t) & 1 for t in range(pr.nT)])
        assert np.array_equal(bits_a[~close], bits_b[~close])


def test_monotone_in_bounds():
    pr = small_problem(N=50, K=3, nT=6, seed=9)
    base = oracle.OracleProblem(pr).edges(with_detail=False)
    pr.model.bounds = tuple(2.0 * np.asarray(pr.model.bounds))
    pr.b = pr.b + 0.5
    loose = oracle.OracleProblem(pr).edges(with_detail=False)
    # enlarging b can only add members, so candidates and bits only grow
    lk = {(int(i), int(j)): int(mk) for i, j, mk in zip(loose["i"], loose["j"], loose["mask"])}
    grew = 0
    for i, j, mk in zip(base["i"], base["j"], base["mask"]):
        other = lk[(int(i), int(j))]
        assert int(mk) & ~other == 0
        grew += bin(other).count("1") - bin(int(mk)).count("1")
    assert grew > 0 and len(lk) >= base["i"].size


def test_translation_invariance():
    pr = small_problem(N=50, K=3, nT=6, seed=13)
    a = oracle.OracleProblem(pr).edges()
    shift = np.array([4.0, -2.0])
    pr.states[:, :2] += shift
    pr.b = pr.b + pr.A @ shift
    b = oracle.OracleProblem(pr).edges()
    assert np.array_equal(a["i"], b["i"]) and np.array_equal(a["j"], b["j"])
    np.testing.assert_allclose(a["rmarg"], b["rmarg"], atol=1e-9)
    np.testing.assert_allclose(a["costs"], b["costs"], rtol=1e-12)


def test_polygon_length_bounds_arc_length():
    """Property 2: sum ||P_{l+1} - P_l|| >= integral of ||x_d'(t)|| (state space)."""
    pr = small_problem(N=40, K=3, nT=6, seed=17)
    op = oracle.OracleProblem(pr)
    e = op.edges()
    xg, wg = np.polynomial.legendre.leggauss(64)
    u = 0.5 * (xg + 1.0)
    m, g = op.m, op.gamma
    for idx in range(0, e["i"].size, 7):
        i, j = int(e["i"][idx]), int(e["j"][idx])
        for t, T in enumerate(pr.T):
            speed2 = np.zeros_like(u)
            for a in range(m):
                P = op.D[t] @ _xi(op, i, j, a)
                for d in range(g):
                    speed2 += pins.t_derivative_at(P, T, d + 1, u) ** 2
            arc = 0.5 * T * float(np.sum(wg * np.sqrt(speed2)))
            assert arc <= e["costs"][idx, t] * (1 + 1e-9) + 1e-12


def test_nearest_vertex_brute_force():
    pr = small_problem(N=300, K=5)
    op = oracle.OracleProblem(pr)
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.uniform(0, 10, 2)
        d = np.sum((pr.states[:, :2] - q) ** 2, axis=1)
        assert op.nearest(q) == int(np.argmin(d))
    # ties go to the lowest id
    pr.states[7, :2] = pr.states[3, :2]
    op = oracle.OracleProblem(pr)
    assert op.nearest(pr.states[3, :2]) == 3


def _brute_paths(N, adj, s, g):
    best = np.inf
    others = [v for v in range(N) if v not in (s, g)]
    if s == g:
        return 0.0
    for r in range(len(others) + 1):
        for mid in itertools.permutations(others, r):
            path = (s,) + mid + (g,)
            c = 0.0
            ok = True
            for u, v in zip(path[:-1], path[1:]):
                if (u, v) not in adj:
                    ok = False
                    break
                c = c + adj[(u, v)]
            if ok:
                best = min(best, c)
    return best


def test_dijkstra_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(60):
        N = int(rng.integers(2, 8))
        adj = {}
        for u in range(N):
            for v in range(N):
                if u != v and rng.uniform() < 0.4:
                    adj[(u, v)] = float(rng.uniform(0.1, 5.0))
        rows = sorted(adj)
        row_off = np.zeros(N + 1, np.int64)
        for u, _ in rows:
            row_off[u + 1] += 1
        row_off = np.cumsum(row_off)
        col = np.array([v for _, v in rows], np.int32)
        w = np.array([adj[e] for e in rows])
        s = int(rng.integers(0, N))
        dist, pred = oracle.dijkstra(N, row_off, col, w, s)
        for g in range(N):
            ref = _brute_paths(N, adj, s, g)
            assert (np.isinf(ref) and np.isinf(dist[g])) or abs(ref - dist[g]) <= 1e-12 * max(1, ref)
            path = oracle.walk(pred, s, g)
            if np.isfinite(ref):
                c = sum(adj[(u, v)] for u, v in zip(path[:-1], path[1:]))
                assert abs(c - ref) <= 1e-12 * max(1, ref)
            else:
                assert path is None


def test_planted_mistake_in_c_oracle_is_caught(tmp_path):
    """Compile copies of plan_oracle.c with plausible slips (right half reading
    the start state; the last free row skipped) and check that the brute-force
    pin rejects each."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "plan_oracle.c")).read()
    slips = {
        "right half reads x_i": ("for (int c = 0; c < g; ++c) sr = sr + h[g + c] * xj[c * m + a];",
                                 "for (int c = 0; c < g; ++c) sr = sr + h[g + c] * xi[c * m + a];"),
        "last free row skipped": ("for (int r = P->poly_off[k]; r < P->poly_off[k + 1]; ++r) {\n                double lim",
                                  "for (int r = P->poly_off[k]; r < P->poly_off[k + 1] - 1; ++r) {\n                double lim"),
        "cost drops a derivative row": ("int drows = (P->cost_mode == 1) ? 1 : g;", "int drows = (P->cost_mode == 1) ? 1 : g - 1;"),
    }
    pr = small_problem(N=40, K=3, nT=6, seed=21)
    good = oracle.OracleProblem(pr).edges()
    for name, (old, new) in slips.items():
        assert old in src, name
        cpath = tmp_path / (name.replace(" ", "_") + ".c")
        cpath.write_text(src.replace(old, new))
        lib = tmp_path / (name.replace(" ", "_") + ".so")
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(cpath), "-o", str(lib), "-lm"], check=True)
        bad = oracle.OracleProblem(pr, lib=oracle.load_variant(str(lib))).edges()
        # the brute-force pin (same comparison as test_pairs_match_brute_force) must fail somewhere
        mism = 0
        mdl = pr.model
        inm = oracle.OracleProblem(pr).membership()
        for idx in range(0, bad["i"].size, 3):
            i, j = int(bad["i"][idx]), int(bad["j"][idx])
            for t, T in enumerate(pr.T):
                fbest = -np.inf
                for k in np.nonzero(inm[i] & inm[j])[0]:
                    lo, hi = pr.poly_off[k], pr.poly_off[k + 1]
                    rm, fm, cost = pins.brute_pair(mdl.m, mdl.gamma, mdl.degree, np.asarray(mdl.bounds), T,
                                                   oracle.OracleProblem(pr).D[t], pr.A[lo:hi], pr.b[lo:hi],
                                                   pr.states[i], pr.states[j])
                    fbest = max(fbest, fm)
                if (abs(bad["rmarg"][idx, t] - rm) > 1e-6 or abs(bad["fmarg"][idx, t] - fbest) > 1e-6
                        or abs(bad["costs"][idx, t] - cost) > 1e-6 * cost):
                    mism += 1
        assert mism > 0, name
