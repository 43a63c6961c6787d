"""Pins for the oracle's coefficient tables (Lemma 1, Theorem 1, Eq. BezDef).

The expected values come from textbook Bezier/Hermite identities and from the
power-basis expansion of the Bernstein form (tests/pins.py), never from the
oracle's own route.  Mutation tests plant plausible mistakes in copies of the
tables and check that at least one pin catches each.
"""
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

from oracle import tables as T_
import pins

CASES = [(2, 3), (2, 5), (3, 5), (3, 7), (2, 7), (1, 3)]
DURATIONS = [0.1, 0.37, 1.0, 2.9]


@pytest.mark.parametrize("gamma,p", CASES)
@pytest.mark.parametrize("T", DURATIONS)
def test_table_pins(gamma, p, T):
    tb = {k: v[0] for k, v in T_.tables(gamma, p, [T]).items()}
    res = pins.all_table_pins(gamma, p, T, tb, seed=gamma * 100 + p)
    for name, worst in res.items():
        assert worst < 1e-9, (name, worst)


MINSNAP_CASES = [(1, 3), (2, 5), (3, 7), (2, 7)]


@pytest.mark.parametrize("gamma,p", MINSNAP_CASES)
@pytest.mark.parametrize("T", DURATIONS)
def test_minsnap_table_pins(gamma, p, T):
    """Minimum-energy interior points: end conditions, hodograph and cost
    identities as for the elevated curve, plus stationarity of the energy in
    every interior point, energy <= the elevated curve's, and the natural
    boundary conditions b^(g+1)(0) = b^(g+1)(T) = 0 at p = 2g+1."""
    tb = {k: v[0] for k, v in T_.tables(gamma, p, [T], "minsnap").items()}
    res = pins.all_table_pins(gamma, p, T, tb, seed=gamma * 100 + p + 7, interior="minsnap")
    assert "minsnap_optimal" in res
    for name, worst in res.items():
        assert worst < 1e-6, (name, worst)


def test_minsnap_equals_elevate_at_minimal_degree():
    for gamma, p in [(2, 3), (3, 5)]:
        a = T_.tables(gamma, p, [0.7], "minsnap")
        b = T_.tables(gamma, p, [0.7], "elevate")
        assert all(np.array_equal(a[k], b[k]) for k in "DHC")


def test_minsnap_pins_catch_planted_mistakes():
    """A perturbed interior row (a plausible slip in the normal equations) is
    caught by the stationarity pin; an elevated-curve table passed off as the
    minimiser is caught too."""
    gamma, p, T = 2, 5, 0.8
    good = {k: v[0] for k, v in T_.tables(gamma, p, [T], "minsnap").items()}
    bad = {k: v.copy() for k, v in good.items()}
    bad["D"][2, 0] *= 1.001
    res = pins.all_table_pins(gamma, p, T, bad, seed=3, interior="minsnap")
    assert res["minsnap_optimal"] > 1e-4
    elev = {k: v[0] for k, v in T_.tables(gamma, p, [T], "elevate").items()}
    res = pins.all_table_pins(gamma, p, T, elev, seed=3, interior="minsnap")
    assert max(res["minsnap_optimal"], res["minsnap_natural"]) > 1e-4


def test_shapes():
    tb = T_.tables(3, 7, [0.5, 1.0])
    assert tb["D"].shape == (2, 8, 6)
    assert tb["H"].shape == (2, 7 + 6 + 5, 6)
    assert tb["C"].shape == (2, 3, 7, 6)
    assert list(T_.reach_row_orders(3, 7)) == [1] * 7 + [2] * 6 + [3] * 5


def test_endpoint_rows_are_exact():
    """Endpoint control points reproduce the states exactly: coefficient 1 on
    x (start at l=0, end at l=p) and exactly 0 elsewhere; so do the endpoint
    hodograph rows k < gamma (b^(k)(0) = xL_k)."""
    for gamma, p in [(2, 5), (3, 7)]:
        for T in DURATIONS:
            tb = T_.tables(gamma, p, [T])
            D, H = tb["D"][0], tb["H"][0]
            e0 = np.zeros(2 * gamma); e0[0] = 1.0
            e1 = np.zeros(2 * gamma); e1[gamma] = 1.0
            assert np.array_equal(D[0], e0) and np.array_equal(D[p], e1)
            row = 0
            for k in range(1, gamma):
                ek = np.zeros(2 * gamma); ek[k] = 1.0
                assert np.array_equal(H[row], ek)
                row += p - k + 1


@pytest.mark.parametrize("gamma,p", [(2, 5), (3, 7)])
def test_exact_symbolic_endpoints(gamma, p):
    """With the exact (rational) tables, sympy's derivative of the Bernstein
    curve hits every boundary condition exactly, and the reach rows equal the
    exact hodograph control points."""
    Tq = Fraction(3, 7)
    ex = T_.exact_tables(gamma, p, float(Tq))
    Tq = Fraction(float(Tq))
    t = sp.symbols("t")
    Ts = sp.Rational(Tq.numerator, Tq.denominator)
    xi = [sp.Rational(v) for v in (3, -2, 5, 7, 1, -4)[:2 * gamma]]
    P = [sum(sp.Rational(ex["D"][l][c].numerator, ex["D"][l][c].denominator) * xi[c] for c in range(2 * gamma))
         for l in range(p + 1)]
    u = t / Ts
    bt = sum(P[l] * sp.binomial(p, l) * u ** l * (1 - u) ** (p - l) for l in range(p + 1))
    for c in range(gamma):
        dc = sp.diff(bt, t, c)
        assert sp.simplify(dc.subs(t, 0) - xi[c]) == 0
        assert sp.simplify(dc.subs(t, Ts) - xi[gamma + c]) == 0
    row = 0
    for k in range(1, gamma + 1):
        dk = sp.expand(sp.diff(bt, t, k))
        Q = [sum(sp.Rational(ex["H"][row + j][c].numerator, ex["H"][row + j][c].denominator) * xi[c]
                 for c in range(2 * gamma)) for j in range(p - k + 1)]
        row += p - k + 1
        hod = sp.expand(sum(Q[j] * sp.binomial(p - k, j) * u ** j * (1 - u) ** (p - k - j) for j in range(p - k + 1)))
        assert sp.simplify(hod - dk) == 0


def _mutations(tb, gamma, p):
    """Plausible slips: sign, dropped term, transposed halves, off-by-one row."""
    out = {}
    D, H, C = tb["D"].copy(), tb["H"].copy(), tb["C"].copy()
    d1 = D.copy(); d1[1, 1] = -d1[1, 1]; out["D sign"] = dict(tb, D=d1)
    d2 = D.copy(); d2[2, 1] = 0.0; out["D dropped term"] = dict(tb, D=d2)
    d3 = D.copy(); d3[:, :gamma], d3[:, gamma:] = D[:, gamma:].copy(), D[:, :gamma].copy(); out["D halves swapped"] = dict(tb, D=d3)
    h1 = H.copy(); h1[p + 1] = H[p + 2]; out["H off-by-one row"] = dict(tb, H=h1)
    h2 = H.copy(); h2[:, 0] = -h2[:, 0]; out["H sign"] = dict(tb, H=h2)
    h3 = H.copy(); h3 *= 1.0 + 1e-3; out["H scale"] = dict(tb, H=h3)
    c1 = C.copy(); c1[1] = C[1] * 2.0; out["C missing factor"] = dict(tb, C=c1)
    c2 = C.copy(); c2[0, 0], c2[0, 1] = C[0, 1].copy(), C[0, 0].copy(); out["C index"] = dict(tb, C=c2)
    c3 = C.copy(); c3[gamma - 1, :, :gamma] = C[gamma - 1, :, gamma:]; out["C transposed operand"] = dict(tb, C=c3)
    return out


@pytest.mark.parametrize("gamma,p", [(2, 5), (3, 7)])
def test_pins_catch_planted_mistakes(gamma, p):
    T = 0.83
    tb = {k: v[0] for k, v in T_.tables(gamma, p, [T]).items()}
    assert max(pins.all_table_pins(gamma, p, T, tb).values()) < 1e-9
    for name, bad in _mutations(tb, gamma, p).items():
        res = pins.all_table_pins(gamma, p, T, bad)
        assert max(res.values()) > 1e-6, (name, res)
