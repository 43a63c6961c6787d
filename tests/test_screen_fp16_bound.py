"""The error bound behind the half-precision screen of the screened pair kernel
(k_pairs_sc): two FP32 reach halves u, w are each rounded to FP16 and summed in
FP16; the kernel rejects a pair only when that sum exceeds the FP32 reach band
widened by KH * (|u| + |w|) + EH (KH = 2^-9, EH = 2^-20), and never when
|u| + |w| > 16384.  The test checks, with exact arithmetic, that the FP16 sum
stays within the derived bound 2^-10 (1 + 2^-11) (|u| + |w|) + 3 * 2^-25 of the
exact sum over magnitudes from the FP16 subnormal range to the guard, that this
bound sits below the kernel's widening, and that the bound is tight enough to
matter (a widening of 2^-11 would not cover the observed error).
"""
import numpy as np

KH = 2.0 ** -9
EH = 2.0 ** -20
MAGH = 16384.0
BOUND_REL = 2.0 ** -10 * (1 + 2.0 ** -11)
BOUND_ABS = 3 * 2.0 ** -25


def fp16_sum(u, w):
    """FP16(FP16(u) + FP16(w)) with one rounding of the exact sum (the sum of
    two FP16 values is exact in float64)."""
    hu = u.astype(np.float16).astype(np.float64)
    hw = w.astype(np.float16).astype(np.float64)
    return (hu + hw).astype(np.float16).astype(np.float64)


def samples(n, seed):
    rng = np.random.default_rng(seed)
    mag_u = np.exp(rng.uniform(np.log(1e-9), np.log(MAGH / 2), n))
    mag_w = np.exp(rng.uniform(np.log(1e-9), np.log(MAGH / 2), n))
    u = (mag_u * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    w = (mag_w * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    # near-cancelling pairs (the margins that decide the screen lie near 1)
    k = n // 4
    w[:k] = (-u[:k].astype(np.float64) + rng.uniform(-2, 2, k)).astype(np.float32)
    return u, w


def test_fp16_sum_within_derived_bound():
    u, w = samples(400_000, 7)
    exact = u.astype(np.float64) + w.astype(np.float64)
    mag = np.abs(u.astype(np.float64)) + np.abs(w.astype(np.float64))
    err = np.abs(fp16_sum(u, w) - exact)
    assert np.all(err <= BOUND_REL * mag + BOUND_ABS), float(np.max(err - BOUND_REL * mag - BOUND_ABS))
    # the kernel's widening is nearly twice the bound
    assert np.all(1.99 * (BOUND_REL * mag + BOUND_ABS) <= KH * mag + EH)
    # and the bound is needed: a widening of 2^-11 (one rounding) is exceeded
    assert np.any(err > 2.0 ** -11 * mag + BOUND_ABS)


def test_fp16_subnormal_and_guard_edges():
    tiny = np.array([2.0 ** -25, 2.0 ** -24, 3 * 2.0 ** -25, 6.1e-5, 6.2e-5, 1e-7], dtype=np.float32)
    u = np.concatenate([tiny, -tiny, np.full(6, MAGH / 2, np.float32), np.full(6, -MAGH / 2, np.float32)])
    w = np.concatenate([tiny[::-1], tiny, np.full(6, MAGH / 2, np.float32) * np.float32(0.999), np.full(6, 1.0, np.float32)])
    exact = u.astype(np.float64) + w.astype(np.float64)
    mag = np.abs(u.astype(np.float64)) + np.abs(w.astype(np.float64))
    s = fp16_sum(u, w)
    assert np.all(np.isfinite(s))  # no overflow below the guard
    assert np.all(np.abs(s - exact) <= BOUND_REL * mag + BOUND_ABS)


def test_screen_rejects_only_certain_failures():
    """The kernel's rule, restated on the CPU: reject iff the FP16 |u + w|
    exceeds 1 + KR * mag + KH * mag + EH with mag <= MAGH.  Every rejected
    pair has an exact |u + w| above 1 (here KR = 0: u, w are taken as exact)."""
    u, w = samples(200_000, 11)
    exact = np.abs(u.astype(np.float64) + w.astype(np.float64))
    mag = np.abs(u.astype(np.float64)) + np.abs(w.astype(np.float64))
    r16 = np.abs(fp16_sum(u, w))
    reject = (r16 > 1.0 + KH * mag + EH) & (mag <= MAGH)
    assert np.all(exact[reject] > 1.0)
    # the screen still rejects most certain failures of moderate magnitude
    moderate = (exact > 1.05) & (mag < 8.0)
    assert np.mean(reject[moderate]) > 0.99
