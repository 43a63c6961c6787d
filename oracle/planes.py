"""FP64 oracle of closestPoint and adjacentHyperplane (Algorithm 2; Sec. III-D,
the separating hyperplane between an MPC node and an obstacle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

closestPoint(v, O) is the Euclidean projection of the point v onto the
convex obstacle O = {z : A z <= b}: the point of O nearest to v.  It is
written out from its definition: the projection lies on some face of O, i.e.
it is the projection of v onto the affine set {z : A_S z = b_S} of an active
set S of at most m facets (S empty when v is in O); every such candidate that
lies in O is a point of O, so the nearest feasible candidate is the
projection.  adjacentHyperplane at that point: h = (v - z) / |v - z|,
l = h . z; O lies in {h . z <= l} and v strictly on the other side.  A point
inside O gets distance 0, z = v and no plane (h = 0, l = 0).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def project(v: np.ndarray, A: np.ndarray, b: np.ndarray, feas_tol: float = 1e-12):
    """(z, distance) of the projection of v onto {z : A z <= b} (None if O is
    empty or no candidate is feasible within feas_tol x scale)."""
    v = np.asarray(v, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64).reshape(-1, v.shape[0])
    b = np.asarray(b, dtype=np.float64)
    m, R = v.shape[0], A.shape[0]
    scale = 1.0 + np.abs(b).max(initial=0.0) + np.abs(v).max()
    if np.all(A @ v - b <= 0.0):
        return v.copy(), 0.0
    best, bd = None, np.inf
    for k in range(1, min(m, R) + 1):
        for S in combinations(range(R), k):
            AS, bS = A[list(S)], b[list(S)]
            G = AS @ AS.T
            if abs(np.linalg.det(G)) < 1e-14 * max(1.0, np.abs(G).max()) ** k:
                continue
            mu = np.linalg.solve(G, AS @ v - bS)
            z = v - AS.T @ mu
            if np.all(A @ z - b <= feas_tol * scale):
                d = float(np.linalg.norm(v - z))
                if d < bd:
                    best, bd = z, d
    return best, bd


def plane(v: np.ndarray, z: np.ndarray, d: float):
    """(h, l) of the separating hyperplane through z, normal toward v."""
    if d <= 0.0:
        return np.zeros_like(v), 0.0
    h = (np.asarray(v, dtype=np.float64) - z) / d
    return h, float(h @ z)


def planes(points: np.ndarray, off, A, b):
    """All (point, obstacle) pairs: closest points [P][n][m], distances [P][n],
    planes [P][n][m+1] (h then l), and per point the nearest obstacle (ties to
    the lowest index; -1 without obstacles) with its distance."""
    points = np.asarray(points, dtype=np.float64)
    P, m = points.shape
    off = np.asarray(off, dtype=np.int64)
    n = off.shape[0] - 1
    A = np.asarray(A, dtype=np.float64).reshape(-1, m)
    b = np.asarray(b, dtype=np.float64)
    Z = np.zeros((P, n, m))
    D = np.zeros((P, n))
    H = np.zeros((P, n, m + 1))
    near = np.full(P, -1, dtype=np.int64)
    nd = np.full(P, np.inf)
    for p in range(P):
        for o in range(n):
            z, d = project(points[p], A[off[o]:off[o + 1]], b[off[o]:off[o + 1]])
            if z is None:
                z, d = np.full(m, np.nan), np.inf
            Z[p, o], D[p, o] = z, d
            h, l = plane(points[p], z, d) if np.isfinite(d) else (np.zeros(m), 0.0)
            H[p, o, :m], H[p, o, m] = h, l
            if d < nd[p]:
                near[p], nd[p] = o, d
    return {"closest": Z, "dist": D, "plane": H, "nearest": near, "nearest_dist": nd}
