"""FP64 oracle of the differentiable refinement objective (one Bezier segment each).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For a degree-p segment with control points P_0..P_p (m axes), duration T and
one free polytope {x : A x <= b}:

  loss = w_snap * J_snap + mu * sum_r phi_delta(margin_r)

  reach margins (Theorem 1 read per axis, every hodograph control point):
      c_k - Q^(k)_{j,a}  and  c_k + Q^(k)_{j,a},   k = 1..gamma, j = 0..p-k,
      Q^(k)_j = p!/(p-k)! T^-k Delta^k P_j
  free margins (Property 1, interior control points):
      b_r - A_r . P_l,   l = 1..p-1
  snap energy: J_snap = int_0^T ||b''''(t)||^2 dt
      = (p!/(p-4)!)^2 T^-7 sum_{j,l} G_jl <Delta^4 P_j, Delta^4 P_l>,
      G_jl = int_0^1 B_j^q B_l^q du = C(q,j) C(q,l) / ((2q+1) C(2q, j+l)), q = p-4
  phi_delta (relaxed log-barrier, C^2): -log m for m >= delta, else
      -log delta + ((m - 2 delta)/delta)^2 / 2 - 1/2.

The gradient with respect to every control point and T is analytic (chain
rule through the linear maps above); parity of it is pinned by central
finite differences and by Gauss-Legendre quadrature of J_snap in the tests.
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np


def phi(m, delta):
    m = np.asarray(m, dtype=np.float64)
    safe = np.maximum(m, delta)
    return np.where(m >= delta, -np.log(safe), -np.log(delta) + 0.5 * ((m - 2 * delta) / delta) ** 2 - 0.5)


def dphi(m, delta):
    m = np.asarray(m, dtype=np.float64)
    safe = np.maximum(m, delta)
    return np.where(m >= delta, -1.0 / safe, (m - 2 * delta) / delta ** 2)


def diff_op(p: int, k: int) -> np.ndarray:
    """Matrix of the k-th forward difference: (p-k+1) x (p+1)."""
    Dk = np.eye(p + 1)
    for _ in range(k):
        Dk = Dk[1:] - Dk[:-1]
    return Dk


def gram(q: int) -> np.ndarray:
    return np.array([[comb(q, j) * comb(q, l) / ((2 * q + 1) * comb(2 * q, j + l)) for l in range(q + 1)]
                     for j in range(q + 1)])


def loss_and_grad(P, T, A, b, nrows, bounds, w_snap=1.0, mu=1.0, delta=0.1):
    """P [S][p+1][m], T [S], A [S][R][m], b [S][R], nrows [S] -> loss [S], dP [S][p+1][m], dT [S]."""
    P = np.asarray(P, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    S, p1, m = P.shape
    p = p1 - 1
    gamma = len(bounds)
    loss = np.zeros(S)
    dP = np.zeros_like(P)
    dT = np.zeros(S)
    for k in range(1, gamma + 1):
        Dk = diff_op(p, k)
        s = factorial(p) / factorial(p - k) * T[:, None, None] ** (-k)
        Q = s * np.einsum("jl,sla->sja", Dk, P)
        for sign in (-1.0, 1.0):
            mg = bounds[k - 1] + sign * Q          # c - Q (sign -1) and c + Q (sign +1)
            loss += mu * phi(mg, delta).sum(axis=(1, 2))
            g = mu * dphi(mg, delta) * sign        # d loss / d Q
            dP += np.einsum("jl,sja->sla", Dk, g * s)
            dT += np.sum(g * Q, axis=(1, 2)) * (-k) / T
    R = A.shape[1]
    valid = np.arange(R)[None, :] < np.asarray(nrows)[:, None]
    for l in range(1, p):
        mg = b - np.einsum("sra,sa->sr", A, P[:, l, :])
        ph = np.where(valid, phi(np.where(valid, mg, 1.0), delta), 0.0)
        loss += mu * ph.sum(axis=1)
        g = np.where(valid, mu * dphi(np.where(valid, mg, 1.0), delta), 0.0)
        dP[:, l, :] -= np.einsum("sr,sra->sa", g, A)
    q = p - 4
    G = gram(q)
    D4 = diff_op(p, 4)
    d4 = np.einsum("jl,sla->sja", D4, P)
    c = (factorial(p) / factorial(p - 4)) ** 2 * T ** (-7)
    quad = np.einsum("jl,sja,sla->s", G, d4, d4)
    J = c * quad
    loss += w_snap * J
    gd4 = w_snap * c[:, None, None] * 2.0 * np.einsum("jl,sla->sja", G, d4)
    dP += np.einsum("jl,sja->sla", D4, gd4)
    dT += w_snap * (-7.0) * J / T
    return loss, dP, dT


def snap_quadrature(P, T, points=4):
    """J_snap by Gauss-Legendre quadrature of ||b''''||^2 (exact for 4 points at p = 7)."""
    P = np.asarray(P, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    S, p1, m = P.shape
    p = p1 - 1
    q = p - 4
    x, w = np.polynomial.legendre.leggauss(points)
    u = 0.5 * (x + 1.0)
    d4 = np.einsum("jl,sla->sja", diff_op(p, 4), P)
    B = np.array([[comb(q, j) * uu ** j * (1 - uu) ** (q - j) for j in range(q + 1)] for uu in u])  # [pts][q+1]
    val = factorial(p) / factorial(p - 4) * np.einsum("uj,sja->sua", B, d4) * T[:, None, None] ** (-4)
    return 0.5 * T * np.einsum("u,su->s", w, np.sum(val ** 2, axis=2))
