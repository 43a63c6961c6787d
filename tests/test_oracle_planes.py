"""Pins for the closestPoint / adjacentHyperplane oracle (oracle/planes.py).
Expected values come from closed forms (axis boxes: clamping; one half-space:
the textbook projection), from dense sampling of the polygon, from the KKT
conditions solved by non-negative least squares, and from planted mistakes."""
import numpy as np
import pytest
from scipy.optimize import nnls

from oracle import planes as OP


def box(lo, hi):
    m = len(lo)
    A = np.concatenate([np.eye(m), -np.eye(m)])
    b = np.concatenate([hi, -np.asarray(lo)])
    return A, b


@pytest.mark.parametrize("m", [2, 3])
def test_box_projection_is_clamping(m):
    rng = np.random.default_rng(m)
    for _ in range(200):
        lo = rng.uniform(-2, 1, size=m)
        hi = lo + rng.uniform(0.1, 2, size=m)
        A, b = box(lo, hi)
        v = rng.uniform(-4, 4, size=m)
        z, d = OP.project(v, A, b)
        zc = np.clip(v, lo, hi)
        assert np.allclose(z, zc, atol=1e-12) and abs(d - np.linalg.norm(v - zc)) < 1e-12


def test_half_space_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(100):
        a = rng.normal(size=2)
        b0 = rng.normal()
        v = rng.normal(size=2) * 3
        z, d = OP.project(v, a[None, :], np.array([b0]))
        s = max(0.0, a @ v - b0)
        assert np.allclose(z, v - s * a / (a @ a), atol=1e-12)
        assert abs(d - s / np.linalg.norm(a)) < 1e-12


def random_polygon(rng, c, r, k):
    th = np.sort(rng.uniform(0, 2 * np.pi, size=k))
    A = np.stack([np.cos(th), np.sin(th)], axis=1)
    b = A @ c + r * rng.uniform(0.5, 1.0, size=k)
    return A, b


@pytest.mark.parametrize("seed", range(4))
def test_against_dense_sampling_and_kkt(seed):
    rng = np.random.default_rng(10 + seed)
    c = rng.uniform(-1, 1, size=2)
    A, b = random_polygon(rng, c, 1.0, int(rng.integers(3, 9)))
    g = np.linspace(-4, 4, 801)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    inside = pts[np.all(pts @ A.T - b <= 0, axis=1)]
    step = g[1] - g[0]
    for _ in range(25):
        v = rng.uniform(-3, 3, size=2)
        z, d = OP.project(v, A, b)
        ds = np.min(np.linalg.norm(inside - v, axis=1))
        assert d <= ds + 1e-12 and ds <= d + 1.5 * step
        assert np.all(A @ z - b <= 1e-9)
        if d > 0:
            act = np.abs(A @ z - b) <= 1e-9
            mu, res = nnls(A[act].T, v - z)     # v - z in the normal cone at z
            assert res < 1e-9 * max(1.0, d)
            h, l = OP.plane(v, z, d)
            assert abs(h @ v - l - d) < 1e-12
            assert np.all(inside @ h - l <= 1e-9)   # the obstacle stays on its side


def test_planted_mistakes_are_caught():
    lo, hi = np.array([0.0, 0.0]), np.array([1.0, 1.0])
    A, b = box(lo, hi)
    v = np.array([2.0, 3.0])                      # diagonal to the corner (1, 1)
    z, d = OP.project(v, A, b)
    assert np.allclose(z, [1.0, 1.0])
    # a sign slip in b projects onto the reflected box
    z2, _ = OP.project(v, A, -b)
    assert z2 is None or not np.allclose(z2, z)
    # active sets of one facet only miss the corner
    orig = OP.combinations

    def singles(it, k):
        return orig(it, k) if k == 1 else iter(())
    OP.combinations = singles
    try:
        z3, _ = OP.project(v, A, b)
    finally:
        OP.combinations = orig
    assert z3 is None or not np.allclose(z3, z)


def test_planes_table_nearest_and_inside():
    A1, b1 = box([0.0, 0.0], [1.0, 1.0])
    A2, b2 = box([3.0, 0.0], [4.0, 1.0])
    off = [0, 4, 8]
    pts = np.array([[0.5, 0.5], [1.4, 0.5], [2.6, 0.5], [2.0, 0.5]])
    r = OP.planes(pts, off, np.concatenate([A1, A2]), np.concatenate([b1, b2]))
    assert r["dist"][0, 0] == 0.0 and r["nearest"][0] == 0
    assert r["nearest"][1] == 0 and r["nearest"][2] == 1
    assert r["nearest"][3] == 0                  # a tie goes to the lower index
    assert np.allclose(r["plane"][1, 0], [1.0, 0.0, 1.0])
