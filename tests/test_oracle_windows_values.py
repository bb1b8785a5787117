"""Pins of the oracle's windows and extended double-double values against
the worked example, brute force, closed forms, exact rational arithmetic
and the paper's theorems."""
import math
import zlib
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


# ---------------------------------------------------------------- windows (def. LRN)

def test_windows_worked_example(golden_worked_example):
    g = golden_worked_example
    s = np.array(g["scales"], dtype=np.int64)
    hk, hs = oracle.concave_cover(s)
    good = oracle.good_mask(s, hk, hs, 6)
    for lam, key, printed in [(0.0, "lambda0", "Q0_printed"), (-3.0, "lambdam3", "Qm3_printed")]:
        kl, N, L, R = oracle.windows(hk, hs, 6, np.array([lam]))
        want = g["derived_by_hand"][key]
        assert (int(kl[0]), float(N[0]), int(L[0]), int(R[0])) == (want["k_lambda"], want["N"], want["l"], want["r"])
        kept = [k for k in range(int(L[0]), int(R[0]) + 1) if good[k]]
        # the printed reduced polynomial keeps a subset of G_p cap [l, r]
        assert set(g[printed]) <= set(kept)
    # at lambda = 0 the printed Q_0 is exactly G_p cap [l, r]
    kl, N, L, R = oracle.windows(hk, hs, 6, np.array([0.0]))
    assert [k for k in range(int(L[0]), int(R[0]) + 1) if good[k]] == g["Q0_printed"]


@pytest.mark.parametrize("seed", range(30))
def test_windows_bruteforce(seed):
    rng = np.random.default_rng(500 + seed)
    d = int(rng.integers(1, 40))
    s = rng.integers(-30, 30, d + 1).astype(np.int64)
    s[rng.uniform(0, 1, d + 1) < 0.2] = oracle.NEG_INF
    if s[0] == oracle.NEG_INF and s[-1] == oracle.NEG_INF:
        s[0] = 0
    hk, hs = oracle.concave_cover(s)
    T = int(rng.integers(1, 25))
    lams = list(rng.normal(0, 4, 30))
    # exact ties: lambda = -slope of a segment; and thresholds landing on integers
    for i in range(hk.size - 1):
        lams.append(-float(Fraction(int(hs[i + 1] - hs[i]), int(hk[i + 1] - hk[i]))))
    lams += [0.0, 1.0, -1.0, 2.5, -0.5]
    lam = np.array(lams)
    kl, N, L, R = oracle.windows(hk, hs, T, lam)
    for i, lm in enumerate(lams):
        ks, Nx, l, r = oracle.windows_bruteforce(hk, hs, T, lm)
        assert (int(L[i]), int(R[i])) == (l, r), (lm, L[i], R[i], l, r)
        assert abs(float(N[i]) - float(Nx)) <= 1e-9 * max(1.0, abs(float(Nx)))
        # k_lambda is unique up to argmax ties: its exact value must reach N
        val = oracle.cover_value(hk, hs, int(kl[i])) + Fraction(lm) * int(kl[i])
        assert abs(float(val - Nx)) <= 1e-12 * max(1.0, abs(float(Nx)))


def test_windows_monotone_in_lambda():
    """l and r are non-decreasing in lambda (App. A: the strip endpoints move
    monotonically with the slope)."""
    c = W.half_circle(1000)
    pre = oracle.precondition(c, 53)
    lam = np.linspace(-40, 40, 4001)
    kl, N, L, R = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    assert np.all(np.diff(L) >= 0) and np.all(np.diff(R) >= 0)
    assert np.all(np.diff(kl) >= 0)


def _avg_window(coef, p, pts):
    pre = oracle.precondition(coef, p)
    lam = oracle.log2_abs(pts.re, pts.im)
    kl, N, L, R = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    return float(np.mean(R - L + 1)), pre


def test_theorem3_sphere_average_bound():
    """Thm. equivAlgo: avg over the sphere of #[l, r] < 1 + 1.9046 sqrt(d T)."""
    rng = np.random.default_rng(21)
    pts = W.sphere_points(20000, rng)
    for coef in [W.unit_square_complex(1000, rng), W.half_circle(1000), W.half_circle(1000, True, rng),
                 W.unit_disk_complex(20000, rng)]:
        avg, pre = _avg_window(coef, 53, pts)
        bound = 1 + 1.9046 * math.sqrt(pre.d * pre.T)
        assert avg < bound, (avg, bound)
    # the half-circle family nearly saturates it (C_3(0) ~ 1.32 asymptotically)
    avg, pre = _avg_window(W.half_circle(1000), 53, pts)
    assert avg > 1.0 * math.sqrt(pre.d * pre.T)


def test_real_line_and_disk_average_bounds():
    rng = np.random.default_rng(22)
    c = W.half_circle(1000)
    avg, pre = _avg_window(c, 53, W.real_circle_points(20000, rng))
    assert avg < 1 + 1.7673 * math.sqrt(pre.d * pre.T)      # eq. compAlgoRe constant
    avg, pre = _avg_window(W.half_circle(1000, True, rng), 53, W.disk_points(20000, rng))
    assert avg < 1 + 2.3141 * math.sqrt(pre.d * pre.T)      # Remark case_disk


def test_one_plus_z_kept_fraction():
    """P = 1 + z (first example of §4.2): both terms are kept exactly when
    |log2|z|| <= T, which on the sphere has probability tanh(T ln 2)."""
    c = W.Coeffs(np.array([1.0, 1.0]))
    p = 1
    rng = np.random.default_rng(23)
    pts = W.sphere_points(1 << 20, rng)
    pre = oracle.precondition(c, p)
    lam = oracle.log2_abs(pts.re, pts.im)
    kl, N, L, R = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    both = np.mean((L == 0) & (R == 1))
    want = math.tanh(pre.T * math.log(2.0))
    sd = math.sqrt(want * (1 - want) / pts.n)
    assert abs(both - want) < 6 * sd + 1e-12, (both, want)


# ---------------------------------------------------------------- values

def _exact_poly(coef, z):
    """sum a_k z^k in exact Gaussian rationals."""
    zr, zi = Fraction(z[0]), Fraction(z[1])
    pr, pi = Fraction(0), Fraction(0)
    n = coef.n_coef
    for k in range(n - 1, -1, -1):
        pr, pi = pr * zr - pi * zi, pr * zi + pi * zr
        sc = Fraction(2) ** int(coef.e2[k]) if coef.e2 is not None else Fraction(1)
        pr += Fraction(float(coef.re[k])) * sc
        pi += (Fraction(float(coef.im[k])) * sc) if coef.im is not None else 0
    return pr, pi


def _abs2_err(got, want):
    return (got[0] - want[0]) ** 2 + (got[1] - want[1]) ** 2


def _S_fraction(Sm, Se, j):
    return Fraction(float(Sm[j])) * Fraction(2) ** int(Se[j])


@pytest.mark.parametrize("seed", range(12))
def test_horner_ref_bruteforce_small_degree(seed):
    rng = np.random.default_rng(700 + seed)
    d = int(rng.integers(0, 9))
    re = rng.normal(0, 1, d + 1) * np.ldexp(1.0, rng.integers(-30, 30, d + 1))
    im = rng.normal(0, 1, d + 1) if seed % 2 else None
    e2 = rng.integers(-2000, 2000, d + 1) if seed % 3 == 0 else None
    coef = W.Coeffs(re, im, e2)
    pts = W.sphere_points(40, rng)
    zim = pts.im if seed % 4 else None
    vals, (Sm, Se), l2M = oracle.horner_ref(coef, pts.re, zim)
    for j in range(pts.n):
        z = (pts.re[j], zim[j] if zim is not None else 0.0)
        want = _exact_poly(coef, z)
        got = vals.fraction(j)
        S = _S_fraction(Sm, Se, j)
        assert _abs2_err(got, want) <= (Fraction(2) ** -100 * S) ** 2, (j, d)
        # S(z) = sum |a_k||z|^k to ~1e-12 relative
        Sx = sum(math.hypot(float(coef.re[k]), float(coef.im[k]) if coef.im is not None else 0.0)
                 * math.hypot(*z) ** k * 2.0 ** (int(coef.e2[k]) if coef.e2 is not None else 0)
                 for k in range(d + 1)) if e2 is None else None
        if Sx is not None and Sx > 0:
            assert abs(float(S) - Sx) <= 1e-12 * Sx


def test_window_sum_exact():
    rng = np.random.default_rng(31)
    d = 30
    coef = W.unit_square_complex(d, rng)
    pts = W.sphere_points(50, rng)
    lo = rng.integers(0, d, pts.n)
    hi = np.minimum(d, lo + rng.integers(0, 12, pts.n))
    good = (rng.uniform(0, 1, d + 1) < 0.7).astype(np.uint8)
    vals = oracle.window_sum(coef, good, pts.re, pts.im, lo, hi)
    for j in range(pts.n):
        zr, zi = Fraction(pts.re[j]), Fraction(pts.im[j])
        pr, pi = Fraction(0), Fraction(0)
        wr, wi = Fraction(1), Fraction(0)
        for k in range(d + 1):
            if lo[j] <= k <= hi[j] and good[k]:
                pr += Fraction(coef.re[k]) * wr - Fraction(coef.im[k]) * wi
                pi += Fraction(coef.re[k]) * wi + Fraction(coef.im[k]) * wr
            wr, wi = wr * zr - wi * zi, wr * zi + wi * zr
        got = vals.fraction(j)
        mag = abs(float(pr)) + abs(float(pi)) + 1e-300
        assert abs(float(got[0] - pr)) + abs(float(got[1] - pi)) <= 2.0 ** -95 * mag * 40


def test_geometric_series_closed_form():
    """sum_{k=0}^{d} z^k = (z^{d+1} - 1)/(z - 1), in exact rationals."""
    d = 1000
    coef = W.geometric(d)
    rng = np.random.default_rng(41)
    r = 1.0 + rng.normal(0, 3e-3, 24)
    t = rng.uniform(0, 2 * math.pi, 24)
    zre, zim = r * np.cos(t), r * np.sin(t)
    vals, (Sm, Se), _ = oracle.horner_ref(coef, zre, zim)
    for j in range(zre.size):
        zr, zi = Fraction(zre[j]), Fraction(zim[j])
        # (z^{d+1} - 1)/(z - 1) with exact complex arithmetic
        pr, pi = Fraction(1), Fraction(0)
        br, bi = zr, zi
        n = d + 1
        while n:
            if n & 1:
                pr, pi = pr * br - pi * bi, pr * bi + pi * br
            br, bi = br * br - bi * bi, 2 * br * bi
            n >>= 1
        nr, ni = pr - 1, pi
        dr, di = zr - 1, zi
        den = dr * dr + di * di
        wr, wi = (nr * dr + ni * di) / den, (ni * dr - nr * di) / den
        got = vals.fraction(j)
        S = _S_fraction(Sm, Se, j)
        assert _abs2_err(got, (wr, wi)) <= (Fraction(2) ** -95 * S) ** 2


def test_chebyshev_closed_form():
    """T_d(cos t) = cos(d t); the monomial coefficients are rounded once to
    53 bits, which moves the value by at most 2^-53 S(x)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 300
    for d in (10, 60, 200):
        coef = W.chebyshev_T(d)
        x = np.cos(np.linspace(0.01, 3.13, 37))
        vals, (Sm, Se), _ = oracle.horner_ref(coef, x, None)
        for j in range(x.size):
            want = mpmath.cos(d * mpmath.acos(mpmath.mpf(float(x[j]))))
            got = vals.fraction(j)
            S = float(_S_fraction(Sm, Se, j))
            err = abs(mpmath.mpf(got[0].numerator) / got[0].denominator - want)
            assert float(err) <= 2.0 ** -52 * S + 1e-300
            assert got[1] == 0


def test_power_minus_one_roots_of_unity():
    for d in (4, 64, 1024):
        coef = W.power_minus_one(d)
        zre = np.array([1.0, -1.0, 0.0, 0.0])
        zim = np.array([0.0, 0.0, 1.0, -1.0])
        vals, _, _ = oracle.horner_ref(coef, zre, zim)
        for j in range(4):
            assert vals.fraction(j) == (0, 0)


def test_zero_point_gives_a0():
    coef = W.Coeffs(np.array([0.25, 3.0, -2.0]), np.array([-1.0, 0.0, 5.0]))
    vals, _, _ = oracle.horner_ref(coef, np.array([0.0]), np.array([0.0]))
    assert vals.fraction(0) == (Fraction(1, 4), Fraction(-1))


# ---------------------------------------------------------------- error theorem (§6)

@pytest.mark.parametrize("family", ["square", "halfcircle_c", "invfact", "lognormal"])
def test_truncation_invariant_and_error_theorem(family):
    """Every dropped term (k outside G_p cap [l, r]) has |a_k z^k| < 2^(-T+1) M
    with M = max_k |a_k z^k| (derivation of eq. err), and
    |P(z) - Q_lambda(z)| < 2^(N - p - 3) (eq. err)."""
    rng = np.random.default_rng(zlib.crc32(family.encode()))
    if family == "square":
        coef = W.unit_square_complex(1000, rng)
        pts = W.sphere_points(300, rng)
    elif family == "halfcircle_c":
        coef = W.half_circle(800, True, rng)
        pts = W.sphere_points(300, rng)
    elif family == "invfact":
        coef = W.inverse_factorial(600)
        pts = W.real_line_points(300, -50, 50, rng)
    else:
        coef = W.lognormal_profile(1500, 0.006, rng)
        pts = W.sphere_points(300, rng)
    p = 53
    pre = oracle.precondition(coef, p)
    vals, (kl, N, L, R) = oracle.fpe_eval(pre, pts.re, pts.im)
    ref, (Sm, Se), l2M = oracle.horner_ref(coef, pts.re, pts.im)
    absa = np.hypot(coef.re, coef.im if coef.im is not None else 0.0)
    with np.errstate(divide="ignore"):
        la = np.log2(absa) + (coef.e2 if coef.e2 is not None else 0)
    lam = oracle.log2_abs(pts.re, pts.im)
    k = np.arange(coef.n_coef)
    for j in range(pts.n):
        kept = np.zeros(coef.n_coef, dtype=bool)
        kept[L[j]:R[j] + 1] = True
        kept &= pre.good.astype(bool)
        lt = la + lam[j] * k
        dropped = ~kept & np.isfinite(lt)
        if dropped.any():
            assert np.max(lt[dropped]) < l2M[j] - pre.T + 1 + 1e-9
        a, b = vals.fraction(j), ref.fraction(j)
        err2 = _abs2_err(a, b)
        bound = Fraction(2) ** int(math.floor(N[j] - p - 3 + 1e-9))
        assert err2 < bound * bound
