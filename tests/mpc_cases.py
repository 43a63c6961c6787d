"""MPC test cases shared by the oracle pins and the GPU parity tests: the
kinematics of a constant input, instances feasible by construction, and the
curve helpers.  Test infrastructure (reads the oracle's tables)."""
from math import factorial

import numpy as np

from oracle import mpc
from oracle import tables as OT


def kin_step(x, u, m, g, dt):
    """x(t + dt) under the constant g-th derivative u, from the Taylor sum of
    each derivative (exact for a polynomial of degree g)."""
    y = np.zeros_like(x)
    for c in range(g):
        for a in range(m):
            s = 0.0
            for j in range(c, g):
                s += x[j * m + a] * dt ** (j - c) / factorial(j - c)
            s += u[a] * dt ** (g - c) / factorial(g - c)
            y[c * m + a] = s
    return y


def instance(seed, m=2, g=2, p=5, H=8, dt=0.1, planes_on=True, bounds=(2.0, 4.0, 30.0)):
    """A reference from the kinematics under small random inputs, x0 = r_0,
    and one plane per segment with a random normal whose offset lies just
    below every control point of the reference segment: the reference
    satisfies the dynamics and every plane row by construction, and its
    reach rows at the bounds used (the pins check it)."""
    rng = np.random.default_rng(seed)
    n = m * g
    x = np.zeros(n)
    x[:m] = rng.uniform(1, 4, size=m)
    x[m:2 * m] = rng.uniform(-0.5, 0.5, size=m)
    ref = [x]
    for k in range(H):
        ref.append(kin_step(ref[-1], rng.normal(0, 0.5, size=m), m, g, dt))
    ref = np.array(ref)
    inst = dict(m=m, g=g, p=p, bounds=bounds[:g], dt=dt, x0=ref[0].copy(), ref=ref,
                Q=np.full(n, 1.0), F=np.full(n, 0.5), R=np.full(m, 0.05), V=np.full(n, 2.0))
    planes = np.zeros((H, m + 1))
    if planes_on:
        for k in range(H):
            h = rng.normal(size=m)
            h /= np.linalg.norm(h)
            planes[k, :m] = h
            Pk = segment_control_points(inst, ref, k)
            planes[k, m] = float((Pk @ h).min()) - rng.uniform(0.0, 0.02)
    inst["planes"] = planes
    inst["keepin_A"], inst["keepin_b"] = None, None
    return inst


def with_keepin(inst, margin=0.01):
    """A keep-in box around every control point of the reference, `margin`
    outside the reference's own extent."""
    m, H = inst["m"], inst["ref"].shape[0] - 1
    pts = np.concatenate([segment_control_points(inst, inst["ref"], k) for k in range(H)])
    lo, hi = pts.min(axis=0) - margin, pts.max(axis=0) + margin
    inst = dict(inst)
    inst["keepin_A"] = np.concatenate([np.eye(m), -np.eye(m)])
    inst["keepin_b"] = np.concatenate([hi, -lo])
    return inst


def bezier_points(ctrl, t):
    """De Casteljau on control points [p+1][m] at parameters t in [0, 1]."""
    out = []
    for s in t:
        pts = np.array(ctrl, dtype=np.float64)
        while pts.shape[0] > 1:
            pts = (1 - s) * pts[:-1] + s * pts[1:]
        out.append(pts[0])
    return np.array(out)


def segment_control_points(inst, x, k):
    m, g, p = inst["m"], inst["g"], inst["p"]
    D = OT.tables(g, p, [inst["dt"]])["D"][0]
    P = np.zeros((p + 1, m))
    for a in range(m):
        xi = np.concatenate([[x[k][c * m + a] for c in range(g)], [x[k + 1][c * m + a] for c in range(g)]])
        P[:, a] = D @ xi
    return P


def objective(inst, x, u):
    Q, F, R, V = inst["Q"], inst["F"], inst["R"], inst["V"]
    ref = inst["ref"]
    H = ref.shape[0] - 1
    J = 0.0
    for k in range(H):
        e = x[k] - ref[k]
        d = x[k + 1] - x[k]
        J += float(e @ (Q * e) + d @ (F * d) + u[k] @ (R * u[k]))
    e = x[H] - ref[H]
    return J + float(e @ (V * e))


def solve(inst):
    keys = ("m", "g", "p", "bounds", "dt", "x0", "ref", "planes", "Q", "F", "R", "V", "keepin_A", "keepin_b")
    return mpc.mpc_qp(*(inst.get(k) for k in keys))
