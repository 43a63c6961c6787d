"""The input generators: deterministic per seed, inside their boxes, with
the stated derivative structure (CPU only)."""
import numpy as np

from paper_2411_13507_gb300 import synth


def test_mpc_references_are_reproducible_and_inside_the_box():
    a = synth.mpc_references(3, 32, 10, 0.1, width=5.0)
    b = synth.mpc_references(3, 32, 10, 0.1, width=5.0)
    assert a.shape == (32, 11, 4) and np.array_equal(a, b)
    assert not np.array_equal(a, synth.mpc_references(4, 32, 10, 0.1, width=5.0))
    pos = a[:, :, :2]
    assert pos.min() >= 0.05 * 5.0 and pos.max() <= 0.95 * 5.0


def test_mpc_references_are_samples_of_cubics_with_their_derivatives():
    """Positions are cubic in time, velocities their derivative: a cubic's
    fourth differences vanish, and Simpson's rule integrates the velocity
    exactly over two steps."""
    dt = 0.1
    r = synth.mpc_references(5, 8, 12, dt, width=5.0)
    pos, vel = r[:, :, :2], r[:, :, 2:]
    d4 = np.diff(pos, n=4, axis=1)
    assert np.abs(d4).max() < 1e-12
    simpson = dt / 3.0 * (vel[:, :-2:2] + 4.0 * vel[:, 1:-1:2] + vel[:, 2::2])
    assert np.allclose(pos[:, 2::2] - pos[:, :-2:2], simpson, atol=1e-12)


def test_triple_integrator_references_carry_accelerations():
    r = synth.mpc_references(6, 4, 8, 0.05, width=5.0, m=3, g=3)
    assert r.shape == (4, 9, 9)
    acc, vel = r[:, :, 6:], r[:, :, 3:6]
    # the velocity of a cubic is quadratic, so Simpson's rule on the acceleration is exact
    simpson = 0.05 / 3.0 * (acc[:, :-2:2] + 4.0 * acc[:, 1:-1:2] + acc[:, 2::2])
    assert np.allclose(vel[:, 2::2] - vel[:, :-2:2], simpson, atol=1e-12)
