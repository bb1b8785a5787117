"""Pins of the oracle's scale, concave cover and G_p against the paper's
worked example, the definitions written out by brute force, and a library
convex-hull routine."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


# ---------------------------------------------------------------- scale (§2.3)

def _scale_by_definition(x: float, y: float, e: int = 0):
    """Smallest integer sigma with |a| < 2^sigma, i.e. 2^(sigma-1) <= |a| <
    2^sigma (eq. sigma), found by comparing exact squares."""
    a2 = (Fraction(x) ** 2 + Fraction(y) ** 2) * Fraction(4) ** e
    if a2 == 0:
        return None
    sig = 0
    while a2 >= Fraction(4) ** sig:
        sig += 1
    while a2 < Fraction(4) ** (sig - 1):
        sig -= 1
    return sig


def test_scale_paper_examples():
    # §2.3: s(3+2i) = 2 = s(3) and s(3+3i) = 3 = s(3) + 1
    s = oracle.scale(np.array([3.0, 3.0, 3.0]), np.array([2.0, 3.0, 0.0]))
    assert list(s) == [2, 3, 2]


def test_scale_real_powers_of_two_and_zero():
    k = np.arange(-1074, 1024, 37)
    x = np.ldexp(1.0, k)
    assert list(oracle.scale(x)) == list(k + 1)        # 2^k has scale k+1
    y = np.nextafter(x, 0.0)
    ok = y > 0
    assert list(oracle.scale(y[ok])) == list(k[ok])    # just below 2^k: scale k
    assert oracle.scale(np.array([0.0]))[0] == oracle.NEG_INF
    assert oracle.scale(np.array([0.0]), np.array([0.0]))[0] == oracle.NEG_INF


def test_scale_complex_bruteforce():
    rng = np.random.default_rng(11)
    n = 3000
    ex = rng.integers(-60, 60, n)
    xr = rng.uniform(-1, 1, n) * np.ldexp(1.0, ex)
    xi = rng.uniform(-1, 1, n) * np.ldexp(1.0, ex + rng.integers(-3, 4, n))
    xi[::7] = 0.0
    xr[::11] = 0.0
    # values on and next to |a| = 2^m exactly: 3/5, 4/5 scaled, and (2^m, 0)
    special_r = [0.6, 0.8, 1.0, np.nextafter(1.0, 0), 3.0, 0.0, 1e-300, 2.0 ** -1070]
    special_i = [0.8, 0.6, 0.0, 0.0, 4.0, -1.0, 1e-300, 2.0 ** -1070]
    xr = np.concatenate([xr, special_r])
    xi = np.concatenate([xi, special_i])
    s = oracle.scale(xr, xi)
    for i in range(xr.size):
        want = _scale_by_definition(float(xr[i]), float(xi[i]))
        got = None if s[i] == oracle.NEG_INF else int(s[i])
        assert got == want, (xr[i], xi[i], got, want)


def test_scale_extended_exponent_shift():
    # eq. exact2pow: s(2^n z) = n + s(z)
    rng = np.random.default_rng(12)
    xr, xi = rng.uniform(-1, 1, 200), rng.uniform(-1, 1, 200)
    e = rng.integers(-5000, 5000, 200)
    assert np.array_equal(oracle.scale(xr, xi, e), oracle.scale(xr, xi) + e)


# ---------------------------------------------------------------- cover (def. EP, §5.1)

def _cover_bruteforce(s):
    """Ecover(k) as the definition: the least concave majorant of E_P on the
    nonzero points, i.e. max over pairs i <= k <= j of the chord value."""
    pts = [(k, int(v)) for k, v in enumerate(s) if v != oracle.NEG_INF]
    ks = [k for k, _ in pts]
    out = {}
    for k in range(ks[0], ks[-1] + 1):
        best = None
        for (i, si) in pts:
            if i > k:
                break
            for (j, sj) in pts:
                if j < k:
                    continue
                if i == j:
                    val = Fraction(si) if i == k else None
                else:
                    val = Fraction(si) + Fraction(sj - si, j - i) * (k - i)
                if val is not None and (best is None or val > best):
                    best = val
        out[k] = best
    return out


def test_cover_worked_example(golden_worked_example):
    g = golden_worked_example
    s = np.array(g["scales"], dtype=np.int64)
    # the table's |a_k| are 2^m exactly, and s(2^m) = m + 1
    assert list(s) == [m + 1 for m in g["abs_log2"]]
    hk, hs = oracle.concave_cover(s)
    assert list(hk) == g["derived_by_hand"]["cover_vertices_k"]
    assert list(hs) == g["derived_by_hand"]["cover_vertices_s"]
    # s(a_k z^k) = s(a_k) - 3k at |z| = 2^-3 (table of §4.1, eq. exact2pow)
    assert [int(v) - 3 * k for k, v in enumerate(s)] == g["scales_lambda_minus3"]


@pytest.mark.parametrize("seed", range(40))
def test_cover_bruteforce_small(seed):
    rng = np.random.default_rng(100 + seed)
    d = int(rng.integers(0, 24))
    s = rng.integers(-20, 20, d + 1).astype(np.int64)
    if seed % 3 == 0:  # plateaus and collinear runs
        s = (rng.integers(-3, 3, d + 1) * 2).astype(np.int64)
    zero = rng.uniform(0, 1, d + 1) < 0.25
    s[zero] = oracle.NEG_INF
    if np.all(s == oracle.NEG_INF):
        s[0] = 0
    hk, hs = oracle.concave_cover(s)
    bf = _cover_bruteforce(s)
    for k, v in bf.items():
        assert oracle.cover_value(hk, hs, k) == v
    # vertices are data points; slopes strictly decreasing
    for k, v in zip(hk, hs):
        assert s[k] == v
    sl = [Fraction(int(hs[i + 1] - hs[i]), int(hk[i + 1] - hk[i])) for i in range(hk.size - 1)]
    assert all(a > b for a, b in zip(sl, sl[1:]))


def test_cover_matches_qhull_large():
    """The upper chain of scipy's convex hull (Qhull) of the points (k, s_k)
    gives the same cover at every integer k."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    for d, gen in [(5000, "disk"), (3000, "halfcircle"), (20000, "lognormal")]:
        if gen == "disk":
            c = W.unit_disk_complex(d, rng)
        elif gen == "halfcircle":
            c = W.half_circle(d)
        else:
            c = W.lognormal_profile(d, 0.004, rng)
        s = oracle.scale(c.re, c.im, c.e2)
        hk, hs = oracle.concave_cover(s)
        pts = np.stack([np.arange(d + 1, dtype=float), s.astype(float)], axis=1)
        # add a point far below so the hull is full-dimensional; its facets are not upper
        low = np.array([[d / 2.0, float(s.min()) - 1e6]])
        hull = spatial.ConvexHull(np.concatenate([pts, low]))
        verts = set(int(v) for v in hull.vertices if v <= d)
        assert set(int(k) for k in hk) <= verts
        for k in verts:
            assert oracle.cover_value(hk, hs, k) == s[k] or oracle.cover_value(hk, hs, k) > s[k]
        up = sorted(k for k in verts if oracle.cover_value(hk, hs, k) == s[k])
        # every Qhull upper vertex lies on our cover and every point is under it
        kk = np.arange(d + 1)
        cov = np.array([float(oracle.cover_value(hk, hs, int(k))) for k in kk])
        assert np.all(s.astype(float) <= cov + 1e-9)
        assert up[0] == 0 and up[-1] == d


def test_cover_degenerate():
    hk, hs = oracle.concave_cover(np.array([5], dtype=np.int64))
    assert list(hk) == [0] and list(hs) == [5]
    s = np.array([oracle.NEG_INF, 3, oracle.NEG_INF, oracle.NEG_INF, 3, oracle.NEG_INF], dtype=np.int64)
    hk, hs = oracle.concave_cover(s)
    assert list(hk) == [1, 4] and list(hs) == [3, 3]
    s = np.array([1, 1, 1, 1, 1], dtype=np.int64)  # flat: collinear points dropped
    hk, hs = oracle.concave_cover(s)
    assert list(hk) == [0, 4]
    with pytest.raises(ValueError):
        oracle.concave_cover(np.array([oracle.NEG_INF] * 3, dtype=np.int64))


# ---------------------------------------------------------------- G_p (eq. threshold)

def test_good_worked_example(golden_worked_example):
    g = golden_worked_example
    s = np.array(g["scales"], dtype=np.int64)
    hk, hs = oracle.concave_cover(s)
    assert list(np.nonzero(oracle.good_mask(s, hk, hs, 6))[0]) == g["derived_by_hand"]["good_T6"]
    # the algorithm's offset T = p + s(d) + 3 = 6 + 4 + 3 = 13
    assert oracle.offset_T(6, 10) == 13
    assert list(np.nonzero(oracle.good_mask(s, hk, hs, 13))[0]) == g["derived_by_hand"]["good_T13"]


@pytest.mark.parametrize("seed", range(20))
def test_good_bruteforce(seed):
    rng = np.random.default_rng(300 + seed)
    d = int(rng.integers(1, 60))
    s = rng.integers(-40, 40, d + 1).astype(np.int64)
    s[rng.uniform(0, 1, d + 1) < 0.2] = oracle.NEG_INF
    s[0] = max(int(s[0]), -40) if s[0] != oracle.NEG_INF else 1
    hk, hs = oracle.concave_cover(s)
    T = int(rng.integers(0, 30))
    g = oracle.good_mask(s, hk, hs, T)
    for k in range(d + 1):
        inside = hk[0] <= k <= hk[-1]
        want = inside and s[k] != oracle.NEG_INF and Fraction(int(s[k])) >= oracle.cover_value(hk, hs, k) - T
        assert bool(g[k]) == bool(want)


def test_good_flat_hull_is_everything():
    # random unit-disk coefficients: every scale is within a few units of the flat cover
    c = W.unit_disk_complex(4000, np.random.default_rng(5))
    pre = oracle.precondition(c, 53)
    assert pre.good.sum() == 4001
    assert pre.T == 53 + 12 + 3
