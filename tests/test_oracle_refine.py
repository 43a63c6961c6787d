"""Pins for the refinement objective's FP64 oracle (loss and gradient)."""
import numpy as np
import pytest

from oracle import refine as R
from paper_2411_13507_gb300 import synth


def batch(S=64, seed=3):
    return synth.refine_segments(seed=seed, S=S)


def test_phi_is_c2_at_delta():
    d = 0.1
    for h in (1e-7, 1e-5):
        lo, hi = d - h, d + h
        assert abs(R.phi(lo, d) - R.phi(hi, d)) < 3 * h / d
        assert abs(R.dphi(lo, d) - R.dphi(hi, d)) < 3 * h / d ** 2
    np.testing.assert_allclose(R.phi(0.5, d), -np.log(0.5))
    # quadratic branch: exact second derivative 1/delta^2
    m = np.array([-0.3, 0.0, 0.05])
    np.testing.assert_allclose((R.dphi(m + 1e-6, d) - R.dphi(m - 1e-6, d)) / 2e-6, 1 / d ** 2, rtol=1e-6)


def test_snap_gram_equals_quadrature():
    rb = batch()
    loss0, _, _ = R.loss_and_grad(rb.P, rb.T, rb.A, rb.b, rb.nrows, rb.bounds, w_snap=1.0, mu=0.0)
    quad = R.snap_quadrature(rb.P, rb.T, points=4)
    np.testing.assert_allclose(loss0, quad, rtol=1e-12)
    # more points change nothing (the integrand is a degree-6 polynomial)
    np.testing.assert_allclose(R.snap_quadrature(rb.P, rb.T, points=8), quad, rtol=1e-12)


def test_snap_zero_on_low_degree_curves():
    """A curve of degree <= 3 (here: elevated cubic) has zero snap."""
    rb = batch(S=8)
    from oracle import tables as OT
    cub = np.zeros_like(rb.P)
    rng = np.random.default_rng(0)
    for s in range(8):
        xi = rng.normal(size=(3, 4))  # per axis: x0, v0, x1, v1
        D = OT.tables(2, 7, [rb.T[s]])["D"][0]   # cubic Hermite elevated to degree 7
        cub[s] = (D @ xi.T)
    l, _, _ = R.loss_and_grad(cub, rb.T, rb.A, rb.b, rb.nrows, rb.bounds, w_snap=1.0, mu=0.0)
    assert np.max(np.abs(l)) < 1e-9


def test_gradient_central_differences():
    rb = batch(S=32, seed=7)
    loss, dP, dT = R.loss_and_grad(rb.P, rb.T, rb.A, rb.b, rb.nrows, rb.bounds)
    rng = np.random.default_rng(1)
    for _ in range(40):
        s = int(rng.integers(0, 32))
        l = int(rng.integers(0, 8))
        a = int(rng.integers(0, 3))
        h = 1e-6 * max(1.0, abs(rb.P[s, l, a]))
        Pp, Pm = rb.P.copy(), rb.P.copy()
        Pp[s, l, a] += h
        Pm[s, l, a] -= h
        fp = R.loss_and_grad(Pp[s:s + 1], rb.T[s:s + 1], rb.A[s:s + 1], rb.b[s:s + 1], rb.nrows[s:s + 1], rb.bounds)[0][0]
        fm = R.loss_and_grad(Pm[s:s + 1], rb.T[s:s + 1], rb.A[s:s + 1], rb.b[s:s + 1], rb.nrows[s:s + 1], rb.bounds)[0][0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - dP[s, l, a]) <= 1e-6 * max(1.0, abs(fd), abs(loss[s]) * 1e-3), (fd, dP[s, l, a])
    for s in range(0, 32, 5):
        h = 1e-7 * rb.T[s]
        Tp, Tm = rb.T.copy(), rb.T.copy()
        Tp[s] += h
        Tm[s] -= h
        fp = R.loss_and_grad(rb.P[s:s + 1], Tp[s:s + 1], rb.A[s:s + 1], rb.b[s:s + 1], rb.nrows[s:s + 1], rb.bounds)[0][0]
        fm = R.loss_and_grad(rb.P[s:s + 1], Tm[s:s + 1], rb.A[s:s + 1], rb.b[s:s + 1], rb.nrows[s:s + 1], rb.bounds)[0][0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - dT[s]) <= 1e-5 * max(1.0, abs(fd)), (fd, dT[s])


def test_planted_mistake_in_gradient_is_caught():
    """A dropped factor in the T-derivative must fail the finite-difference pin."""
    rb = batch(S=4, seed=9)
    loss, dP, dT = R.loss_and_grad(rb.P, rb.T, rb.A, rb.b, rb.nrows, rb.bounds)
    bad = dT * 0.5
    s = 0
    h = 1e-7 * rb.T[s]
    Tp, Tm = rb.T.copy(), rb.T.copy()
    Tp[s] += h
    Tm[s] -= h
    fp = R.loss_and_grad(rb.P[:1], Tp[:1], rb.A[:1], rb.b[:1], rb.nrows[:1], rb.bounds)[0][0]
    fm = R.loss_and_grad(rb.P[:1], Tm[:1], rb.A[:1], rb.b[:1], rb.nrows[:1], rb.bounds)[0][0]
    fd = (fp - fm) / (2 * h)
    assert abs(fd - dT[0]) <= 1e-5 * max(1.0, abs(fd))
    assert abs(fd - bad[0]) > 1e-3 * max(1.0, abs(fd))


def test_initial_segments_are_strictly_inside():
    """The generator keeps every control point inside its polytope (finite barrier)."""
    rb = batch(S=256)
    for l in range(8):
        mg = rb.b - np.einsum("sra,sa->sr", rb.A, rb.P[:, l, :])
        valid = np.arange(rb.A.shape[1])[None, :] < rb.nrows[:, None]
        assert np.all(mg[valid] > 0)
