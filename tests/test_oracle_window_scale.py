"""Pins of the oracle's window scale S_w(z) = sum over k in G_p cap [l, r] of
|a_k| |z|^k, the second output of ``oracle.window_sum(..., with_S=True)``.

S_w is the tolerance scale of every all-points parity check (the value
|P_gpu - Q| must stay below 2^-50 S_w), so a slip in it (a wrong good-mask skip,
a wrong |z|^l factor, a dropped term) would loosen every one of those checks.
Here it is compared with its definition evaluated term by term in 200-bit
arithmetic (mpmath), on small inputs chosen so that each of those slips
changes the value: random good masks, windows that start above k = 0, |z|
far from 1 on both sides, coefficients with binary exponents far outside the
FP64 range, real and complex operands, and long runs of skipped terms.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

mpmath = pytest.importorskip("mpmath")


def s_exact(coef, good, zr, zi, lo, hi):
    """sum_{k in [lo, hi], good[k]} |a_k| |z|^k with a_k = (re + i im) 2^e2, in 200-bit arithmetic."""
    with mpmath.workprec(200):
        az = mpmath.hypot(mpmath.mpf(float(zr)), mpmath.mpf(0.0 if zi is None else float(zi)))
        tot = mpmath.mpf(0)
        for k in range(lo, hi + 1):
            if good is not None and not good[k]:
                continue
            a = mpmath.hypot(mpmath.mpf(float(coef.re[k])), mpmath.mpf(0.0 if coef.im is None else float(coef.im[k])))
            if coef.e2 is not None:
                a = mpmath.ldexp(a, int(coef.e2[k]))
            tot += a * az ** k
        return tot


def rel_err(Sm, Se, want):
    with mpmath.workprec(200):
        got = mpmath.ldexp(mpmath.mpf(float(Sm)), int(Se))
        if want == 0:
            return 0.0 if got == 0 else math.inf
        return float(abs(got - want) / want)


def check(coef, good, zr, zi, lo, hi, tol=1e-12):
    _, (Sm, Se) = oracle.window_sum(coef, good, zr, zi, lo, hi, with_S=True)
    for j in range(len(zr)):
        want = s_exact(coef, good, zr[j], None if zi is None else zi[j], int(lo[j]), int(hi[j]))
        e = rel_err(Sm[j], Se[j], want)
        assert e <= tol, f"point {j}: S relative error {e:.3g} (window [{lo[j]}, {hi[j]}])"


@pytest.mark.parametrize("real_coef", [False, True])
@pytest.mark.parametrize("real_pts", [False, True])
def test_window_scale_random_masks(real_coef, real_pts):
    """d = 30: random 0/1 masks, random windows with l > 0, |z| = 2^-20 .. 2^20."""
    rng = np.random.default_rng(31 + 2 * real_coef + real_pts)
    d = 30
    c = W.unit_square_complex(d, rng)
    coef = W.Coeffs(c.re, None if real_coef else c.im)
    good = (rng.uniform(size=d + 1) < 0.6).astype(np.uint8)
    n = 24
    mod = 2.0 ** rng.uniform(-20, 20, n)
    mod[:3] = [2.0 ** 20, 2.0 ** -20, 1.0]
    ph = rng.uniform(0, 2 * math.pi, n)
    zr = mod * np.cos(ph)
    zi = None if real_pts else mod * np.sin(ph)
    lo = rng.integers(1, 12, n)
    hi = rng.integers(15, d + 1, n)
    check(coef, good, zr, zi, lo, hi)


def test_window_scale_extended_exponents():
    """Coefficients 2^e2 with |e2| up to 3000 (far outside FP64), |z| near 1 and 2^+-7."""
    rng = np.random.default_rng(77)
    d = 28
    c = W.unit_square_complex(d, rng)
    e2 = rng.integers(-3000, 3000, d + 1).astype(np.int64)
    e2[5:12] = rng.integers(-40, 40, 7)  # a cluster of comparable terms
    coef = W.Coeffs(c.re, c.im, e2)
    good = np.ones(d + 1, dtype=np.uint8)
    good[rng.integers(0, d + 1, 6)] = 0
    n = 16
    mod = 2.0 ** rng.uniform(-7, 7, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    lo = rng.integers(0, 8, n)
    hi = rng.integers(10, d + 1, n)
    check(coef, good, mod * np.cos(ph), mod * np.sin(ph), lo, hi)


def test_window_scale_long_skipped_runs():
    """Runs of up to ~2400 skipped terms (bad or zero coefficients) between kept
    ones at |z| < 1: the running sum is multiplied by |z| at every skipped step
    and must stay normalised (|z|^2400 is far below the FP64 range)."""
    rng = np.random.default_rng(5)
    d = 2600
    c = W.unit_disk_complex(d, rng)
    re, im = c.re.copy(), c.im.copy()
    re[40:1500] = 0.0  # zero coefficients
    im[40:1500] = 0.0
    good = np.ones(d + 1, dtype=np.uint8)
    good[1500:2500] = 0  # bad coefficients
    coef = W.Coeffs(re, im)
    mod = np.array([0.5, 0.7, 0.9, 1.0, 1.1])
    ph = np.array([0.3, 1.1, 2.0, 2.9, 4.0])
    lo = np.array([0, 3, 30, 39, 0])
    hi = np.array([d, d, 2550, d, 2520])
    check(coef, good, mod * np.cos(ph), mod * np.sin(ph), lo, hi)


def test_window_scale_equals_full_scale():
    """Over [0, d] with every k good, S_w is the full S(z) that horner_ref
    computes by its own loop."""
    rng = np.random.default_rng(9)
    d = 300
    coef = W.unit_disk_complex(d, rng)
    pts = W.sphere_points(64, rng)
    lo = np.zeros(64, dtype=np.int64)
    hi = np.full(64, d, dtype=np.int64)
    _, (Sm, Se) = oracle.window_sum(coef, np.ones(d + 1, dtype=np.uint8), pts.re, pts.im, lo, hi, with_S=True)
    _, (Hm, He), _ = oracle.horner_ref(coef, pts.re, pts.im)
    a = np.ldexp(Sm, (Se - He).astype(np.int32))
    assert np.all(np.abs(a - Hm) <= 1e-12 * Hm)


def test_window_scale_empty_window():
    """An empty window (hi < lo) has S_w = 0."""
    coef = W.unit_square_complex(10, np.random.default_rng(0))
    _, (Sm, Se) = oracle.window_sum(coef, None, np.array([0.5]), np.array([0.5]), np.array([3]), np.array([2]),
                                    with_S=True)
    assert Sm[0] == 0.0
