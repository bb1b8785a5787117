"""Pins of ``oracle.window_sum_fp64``, Algorithm A_p's window sum as a plain
FP64 CPU program (the CPU baseline that bench.py times).  Its value is compared
with the exact rational window sum: FP64 Horner over L terms has error at most
about 2 L u S_w (u = 2^-53, S_w the window's sum of |a_k||z|^k), so the check
is |value - exact| <= 4 L u S_w (with S_w replaced by the larger
sum of |Re a_k| + |Im a_k| times |Re z^k| + |Im z^k|, at most 2 S_w); a dropped term, a wrong power of z, a wrong
good-mask skip or a wrong exponent frame would exceed that by far.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


def exact(coef, good, zr, zi, lo, hi):
    """(re, im) of the window sum as rationals, and S_w as a rational bound
    (|a|_1 / sqrt 2 <= |a|: the L1 norm of each term over sqrt 2 is below S_w's term)."""
    zR, zI = Fraction(float(zr)), Fraction(0.0 if zi is None else float(zi))
    pr, pi = Fraction(0), Fraction(0)
    wr, wi = Fraction(1), Fraction(0)
    S = Fraction(0)
    for k in range(hi + 1):
        if k >= lo and (good is None or good[k]):
            sc = Fraction(2) ** int(coef.e2[k]) if coef.e2 is not None else Fraction(1)
            ar = Fraction(float(coef.re[k])) * sc
            ai = (Fraction(float(coef.im[k])) * sc) if coef.im is not None else Fraction(0)
            pr += ar * wr - ai * wi
            pi += ar * wi + ai * wr
            S += (abs(ar) + abs(ai)) * (abs(wr) + abs(wi))  # >= |a_k| |z|^k
        wr, wi = wr * zR - wi * zI, wr * zI + wi * zR
    return pr, pi, S


def check(coef, good, zr, zi, lo, hi):
    v = oracle.window_sum_fp64(coef, good, zr, zi, lo, hi)
    for j in range(len(zr)):
        er, ei, S = exact(coef, good, zr[j], None if zi is None else zi[j], int(lo[j]), int(hi[j]))
        gr, gi = v.fraction(j)
        L = max(1, int(hi[j]) - int(lo[j]) + 1)
        err2 = (gr - er) ** 2 + (gi - ei) ** 2
        # S (an L1 form) is at most 2 S_w: the bound 4 L u S_w is checked as 2 L u S
        assert err2 <= (Fraction(2 * L) * Fraction(2) ** -53 * S) ** 2, j


@pytest.mark.parametrize("real_pts", [False, True])
def test_fp64_window_sum_random(real_pts):
    rng = np.random.default_rng(101 + real_pts)
    d = 40
    coef = W.unit_square_complex(d, rng)
    good = (rng.uniform(size=d + 1) < 0.7).astype(np.uint8)
    n = 20
    mod = 2.0 ** rng.uniform(-6, 6, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    zr = mod * np.cos(ph)
    zi = None if real_pts else mod * np.sin(ph)
    lo = rng.integers(0, 15, n)
    hi = rng.integers(15, d + 1, n)
    check(coef, good, zr, zi, lo, hi)


def test_fp64_window_sum_extended_exponents():
    """Exponents far outside FP64 (|e2| up to 2000): the exponent frame and the
    renormalisation of the running sum are exercised."""
    rng = np.random.default_rng(7)
    d = 30
    c = W.unit_disk_complex(d, rng)
    e2 = (np.arange(d + 1) * 70 - 1000).astype(np.int64)  # terms grow by 2^70 per index
    coef = W.Coeffs(c.re, c.im, e2)
    n = 12
    mod = 2.0 ** rng.uniform(-75, -65, n)  # |a_k z^k| varies over a few hundred bits across the window
    ph = rng.uniform(0, 2 * math.pi, n)
    check(coef, None, mod * np.cos(ph), mod * np.sin(ph), np.zeros(n, np.int64), np.full(n, d, np.int64))


def test_fp64_restatement_end_to_end():
    """fpe_eval_fp64 agrees with the extended double-double fpe_eval to the
    FP64 rounding of its window sums (2^-40 S on this workload)."""
    wl = W.unit_square_d1000(n_points=256)
    pre = oracle.precondition(wl.coeffs, 53)
    a, _ = oracle.fpe_eval_fp64(pre, wl.points.re, wl.points.im)
    b, _ = oracle.fpe_eval(pre, wl.points.re, wl.points.im)
    _, (Sm, Se), _ = oracle.horner_ref(wl.coeffs, wl.points.re, wl.points.im)
    sc = lambda m, e: np.ldexp(m, np.clip(e - Se, -2000, 2000).astype(np.int32))
    dr = sc(a.re_hi, a.e) + sc(a.re_lo, a.e) - sc(b.re_hi, b.e) - sc(b.re_lo, b.e)
    di = sc(a.im_hi, a.e) + sc(a.im_lo, a.e) - sc(b.im_hi, b.e) - sc(b.im_lo, b.e)
    assert np.all(np.hypot(dr, di) <= 2.0 ** -40 * Sm)
