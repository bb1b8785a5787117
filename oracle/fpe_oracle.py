"""CPU ORACLE for fast polynomial evaluation (FPE) -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It shares no code with the CUDA path and imports
nothing from it.

Each function restates one step of Algorithm A_p (§4.3) in plain form, in
the paper's notation:

* ``scale``          -- s(a) = 1 + floor(log2 |a|), s(0) = -inf (eq. dsz, §2.3),
                        exact for real and complex FP64 (with an optional
                        extra binary exponent per value).
* ``concave_cover``  -- the concave cover of E_P(k) = s(a_k) (def. EP), built
                        as in §5.1: sort the scales decreasing (ties by
                        increasing k), then extend the cover left or right
                        one point at a time with a binary search over the
                        lines of its segments (Lemma of §5.1 and its proof).
* ``good_mask``      -- G_p = {k : s(a_k) >= Ecover(k) - p - s(d) - 3}
                        (eq. threshold), by exact integer arithmetic.
* ``windows``        -- per point: lambda = log2|z| (eq. defLambda), k_lambda =
                        argmax(Ecover + lambda Id) (ties: leftmost vertex), N =
                        Ecover(k_lambda) + lambda k_lambda (eq. defN) and [l, r],
                        the largest integer interval where Ecover(k) + lambda k
                        >= N - p - s(d) - 3 (def. LRN).  FP64 throughout, as the
                        GPU path decides it; a boundary within 1e-6 of the
                        threshold is re-decided in exact rational arithmetic
                        for the given FP64 lambda.
* ``horner_ref``     -- P(z) by Horner over all d+1 terms in extended
                        double-double (C, ``ext_dd.c``), with S(z) = sum
                        |a_k||z|^k and log2 max_k |a_k z^k|.
* ``window_sum``     -- Q_lambda(z) = sum_{k in G_p cap [l, r]} a_k z^k
                        (eq. reducedQlambda) in extended double-double.
* ``fpe_eval``       -- Algorithm A_p end to end: windows, then window_sum.
* ``window_sum_fp64``, ``fpe_eval_fp64`` -- the same with the window's Horner
                        steps in plain FP64 (a CPU baseline for timing, pinned
                        by exact sums, not a reference value).

Readings where the paper is silent:
  p counts significand bits (53 for FP64, 24 for FP32); T = p + s(d) + 3 with
  d the index of the last nonzero coefficient; the cover is taken over the
  nonzero coefficients only, on [v, d] with v the first nonzero index; its
  vertex list keeps strict vertices only (slopes strictly decreasing);
  threshold comparisons are inclusive; for d = 0 the window is {0}.
"""
from __future__ import annotations

import ctypes
import math
import os
from fractions import Fraction
from typing import Optional, Tuple

import numpy as np

NEG_INF = np.iinfo(np.int64).min  # stands for s(0) = -infinity


# ----------------------------------------------------------------------------
# scale  (eq. dsz / eq. sz, §2.3)
# ----------------------------------------------------------------------------

def _exact_abs2_ge_pow4(x: float, y: float, m: int) -> bool:
    """Exact test x^2 + y^2 >= 2^(2m) with Python rationals."""
    fx, fy = Fraction(x), Fraction(y)
    return fx * fx + fy * fy >= Fraction(2) ** (2 * m)


def scale(re: np.ndarray, im: Optional[np.ndarray] = None,
          e2: Optional[np.ndarray] = None) -> np.ndarray:
    """s(a) = 1 + floor(log2|a|) for a = (re + i im) 2^e2; NEG_INF for a = 0.

    Real a: frexp gives |a| = m 2^f with m in [0.5, 1), so 2^(f-1) <= |a| < 2^f
    and s = f (eq. sigma).  Complex a: with f = max of the two frexp exponents,
    2^(f-1) <= |a| < 2^f sqrt(2), so s is f or f + 1 (eq. sz), and it is f + 1
    exactly when re^2 + im^2 >= 2^(2f).  That test is taken in FP64 when it is
    clear by a wide margin and in exact rationals otherwise."""
    re = np.asarray(re, dtype=np.float64)
    n = re.shape[0]
    out = np.full(n, NEG_INF, dtype=np.int64)
    if im is None:
        nz = re != 0.0
        _, f = np.frexp(re)
        out[nz] = f[nz]
    else:
        im = np.asarray(im, dtype=np.float64)
        nz = (re != 0.0) | (im != 0.0)
        _, fr = np.frexp(re)
        _, fi = np.frexp(im)
        fr = np.where(re != 0.0, fr, np.iinfo(np.int32).min)
        fi = np.where(im != 0.0, fi, np.iinfo(np.int32).min)
        f = np.maximum(fr, fi).astype(np.int64)
        # scaled squares: |a|^2 / 2^(2f) in [1/4, 2)
        fs = np.where(nz, f, 0)
        xs = np.ldexp(re, (-fs).astype(np.int32))
        ys = np.ldexp(im, (-fs).astype(np.int32))
        q = xs * xs + ys * ys
        up = q >= 1.0
        near = nz & (np.abs(q - 1.0) < 1e-9)
        for i in np.nonzero(near)[0]:
            up[i] = _exact_abs2_ge_pow4(float(re[i]), float(im[i]), int(f[i]))
        s = f + up.astype(np.int64)
        out[nz] = s[nz]
    if e2 is not None:
        e2 = np.asarray(e2, dtype=np.int64)
        nzm = out != NEG_INF
        out[nzm] = out[nzm] + e2[nzm]
    return out


def scale_of_int(n: int) -> int:
    """s(n) for a positive integer n: 1 + floor(log2 n) = its bit length."""
    return int(n).bit_length()


def offset_T(p: int, d: int) -> int:
    """T = p + s(d) + 3 (Alg. A_p; eq. threshold), d = degree.
    For d = 0 (a constant) the window is always {0}; s(0) is taken as 0."""
    return p + (scale_of_int(d) if d >= 1 else 0) + 3


# ----------------------------------------------------------------------------
# concave cover  (def. EP; §5.1 construction)
# ----------------------------------------------------------------------------

def _line_at(ka: int, sa: int, kb: int, sb: int, x: int) -> Fraction:
    """Value at abscissa x of the line through (ka, sa) and (kb, sb)."""
    return Fraction(sa) + Fraction(sb - sa, kb - ka) * (x - ka)


def _s_le_line(s: int, ka: int, sa: int, kb: int, sb: int, x: int) -> bool:
    """s <= value at x of the line through (ka, sa), (kb, sb) (ka < kb), exactly:
    s (kb - ka) <= sa (kb - ka) + (sb - sa)(x - ka)."""
    return s * (kb - ka) <= sa * (kb - ka) + (sb - sa) * (x - ka)


def concave_cover(s: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Vertices (k_i, s_i) of the concave cover of E_P over the nonzero
    coefficients (s[k] != NEG_INF), left to right, strict vertices only.

    §5.1: sort the scales decreasingly, ties by increasing k.  The cover E_n
    of the first n+1 sorted points lives on [l_n, r_n].  A new point (k, s)
    with k inside (l_n, r_n) lies under E_n (its scale is at most min E_n).
    Otherwise, say k < l_n: the lines Sigma_j of the segments of E_n, left to
    right, take increasing values y_j at x = k; a binary search finds the j
    with s in (y_{j-1}, y_j], and E_{n+1} is the segment from (k, s) to the
    left end of Sigma_j's segment followed by E_n from there on.  The case
    k > r_n is the mirror image."""
    s = np.asarray(s, dtype=np.int64)
    ks = np.nonzero(s != NEG_INF)[0]
    if ks.size == 0:
        raise ValueError("zero polynomial")
    # sort by decreasing scale, ties by increasing index (stable sort on -s)
    order = ks[np.argsort(-s[ks], kind="stable")]
    n = order.size
    # vertices live in buf[head..tail]; each insertion moves head or tail by 1
    bk = [0] * (2 * n + 1)
    bs = [0] * (2 * n + 1)
    head = tail = n
    bk[n], bs[n] = int(order[0]), int(s[order[0]])
    for idx in order[1:]:
        k, sk = int(idx), int(s[idx])
        lk, rk = bk[head], bk[tail]
        if lk < k < rk:
            continue  # E_{n+1} = E_n
        if k < lk:
            nseg = tail - head
            if nseg == 0:
                head -= 1
                bk[head], bs[head] = k, sk
                continue
            # smallest j in [0, nseg) with sk <= y_j ; nseg if none
            lo, hi = 0, nseg
            while lo < hi:
                mid = (lo + hi) // 2
                a = head + mid
                if _s_le_line(sk, bk[a], bs[a], bk[a + 1], bs[a + 1], k):
                    hi = mid
                else:
                    lo = mid + 1
            keep = head + lo if lo < nseg else tail  # left end of Sigma_j, or r_n
            head = keep - 1
            bk[head], bs[head] = k, sk
        else:  # k > rk: mirror image, segments enumerated right to left
            nseg = tail - head
            if nseg == 0:
                tail += 1
                bk[tail], bs[tail] = k, sk
                continue
            lo, hi = 0, nseg
            while lo < hi:
                mid = (lo + hi) // 2
                b = tail - mid
                if _s_le_line(sk, bk[b - 1], bs[b - 1], bk[b], bs[b], k):
                    hi = mid
                else:
                    lo = mid + 1
            keep = tail - lo if lo < nseg else head
            tail = keep + 1
            bk[tail], bs[tail] = k, sk
    vk = bk[head:tail + 1]
    vs = bs[head:tail + 1]
    # canonical form: drop vertices collinear with their neighbours
    ck, cs = [vk[0]], [vs[0]]
    for i in range(1, len(vk)):
        ck.append(vk[i])
        cs.append(vs[i])
        while len(ck) >= 3:
            (k0, s0), (k1, s1), (k2, s2) = (ck[-3], cs[-3]), (ck[-2], cs[-2]), (ck[-1], cs[-1])
            if (s1 - s0) * (k2 - k1) == (s2 - s1) * (k1 - k0):
                del ck[-2], cs[-2]
            else:
                break
    return np.array(ck, dtype=np.int64), np.array(cs, dtype=np.int64)


def cover_value(hk: np.ndarray, hs: np.ndarray, k: int) -> Fraction:
    """Ecover(k) exactly (piecewise-linear interpolation of the vertices)."""
    i = int(np.searchsorted(hk, k, side="right")) - 1
    if i >= hk.size - 1:
        if k == hk[-1]:
            return Fraction(int(hs[-1]))
        raise ValueError("k outside the cover")
    if k < hk[0]:
        raise ValueError("k outside the cover")
    return _line_at(int(hk[i]), int(hs[i]), int(hk[i + 1]), int(hs[i + 1]), k)


# ----------------------------------------------------------------------------
# good indices  (Alg. A_p, eq. threshold)
# ----------------------------------------------------------------------------

def good_mask(s: np.ndarray, hk: np.ndarray, hs: np.ndarray, T: int) -> np.ndarray:
    """G_p as a 0/1 mask over [0, n_coef): s_k >= Ecover(k) - T, exactly.
    On the segment [k_i, k_{i+1}] (dk = k_{i+1} - k_i > 0, ds = s_{i+1} - s_i):
    s_k - s_i + T >= ds (k - k_i)/dk  <=>  (s_k - s_i + T) dk >= ds (k - k_i)."""
    s = np.asarray(s, dtype=np.int64)
    n = s.shape[0]
    g = np.zeros(n, dtype=np.uint8)
    k = np.arange(n, dtype=np.int64)
    inside = (k >= hk[0]) & (k <= hk[-1]) & (s != NEG_INF)
    kk = k[inside]
    seg = np.searchsorted(hk, kk, side="right") - 1
    seg = np.minimum(seg, hk.size - 2) if hk.size >= 2 else np.zeros_like(seg)
    if hk.size == 1:
        g[kk] = 1  # single coefficient
        return g
    ki, si = hk[seg], hs[seg]
    dk = hk[seg + 1] - ki
    ds = hs[seg + 1] - si
    lhs = (s[kk] - si + T).astype(object) * dk.astype(object)
    rhs = ds.astype(object) * (kk - ki).astype(object)
    g[kk] = (lhs >= rhs).astype(np.uint8)
    return g


# ----------------------------------------------------------------------------
# windows  (Alg. A_p; eq. defN, def. LRN)
# ----------------------------------------------------------------------------

def log2_abs(zre: np.ndarray, zim: Optional[np.ndarray]) -> np.ndarray:
    """lambda = log2|z| (eq. defLambda) in FP64; -inf at z = 0."""
    with np.errstate(divide="ignore"):
        if zim is None:
            return np.log2(np.abs(zre))
        return np.log2(np.hypot(zre, zim))


def _f_exact(hk, hs, k: int, lam: float) -> Fraction:
    return cover_value(hk, hs, k) + Fraction(lam) * k


def windows(hk: np.ndarray, hs: np.ndarray, T: int, lam: np.ndarray,
            chunk: int = 1 << 16):
    """Per point: (k_lambda, N, l, r) with l > r marking 'no window' (z = 0).

    k_lambda: the vertex maximising s_i + lambda k_i, leftmost on ties.
    l: if every vertex left of k_lambda is >= N - T, l = k_0; else on the
       segment (j, j+1) right after the last vertex j < k_lambda below the
       threshold, l = ceil(k_j + (N - T - f_j) dk / (f_{j+1} - f_j)).
    r: the mirror image on the right branch."""
    lam = np.asarray(lam, dtype=np.float64)
    npts = lam.shape[0]
    kl = np.zeros(npts, dtype=np.int64)
    N = np.zeros(npts)
    L = np.zeros(npts, dtype=np.int64)
    R = np.full(npts, -1, dtype=np.int64)
    hkf = hk.astype(np.float64)
    hsf = hs.astype(np.float64)
    h = hk.size
    for c0 in range(0, npts, chunk):
        c1 = min(npts, c0 + chunk)
        lm = lam[c0:c1]
        fin = np.isfinite(lm)
        lmf = np.where(fin, lm, 0.0)
        f = hsf[None, :] + lmf[:, None] * hkf[None, :]  # (m, h)
        istar = np.argmax(f, axis=1)  # first maximum: leftmost on ties
        Nv = f[np.arange(c1 - c0), istar]
        thr = Nv - T
        below = f < thr[:, None]
        idx = np.arange(h)[None, :]
        # left: last vertex j < istar with f_j < thr
        lmask = below & (idx < istar[:, None])
        has_l = lmask.any(axis=1)
        jl = np.where(has_l, h - 1 - np.argmax(lmask[:, ::-1], axis=1), 0)
        # right: first vertex j > istar with f_j < thr
        rmask = below & (idx > istar[:, None])
        has_r = rmask.any(axis=1)
        jr = np.where(has_r, np.argmax(rmask, axis=1), h - 1)
        Lv = np.full(c1 - c0, hk[0], dtype=np.int64)
        Rv = np.full(c1 - c0, hk[-1], dtype=np.int64)
        rows = np.nonzero(has_l)[0]
        if rows.size:
            j = jl[rows]
            fj, fj1 = f[rows, j], f[rows, j + 1]
            x = hkf[j] + (thr[rows] - fj) * (hkf[j + 1] - hkf[j]) / (fj1 - fj)
            Lv[rows] = np.minimum(np.ceil(x), hkf[j + 1]).astype(np.int64)
        rows = np.nonzero(has_r)[0]
        if rows.size:
            j = jr[rows]
            fj, fjm = f[rows, j], f[rows, j - 1]
            x = hkf[j - 1] + (thr[rows] - fjm) * (hkf[j] - hkf[j - 1]) / (fj - fjm)
            Rv[rows] = np.maximum(np.floor(x), hkf[j - 1]).astype(np.int64)
        kl[c0:c1] = hk[istar]
        N[c0:c1] = Nv
        L[c0:c1] = np.where(fin, Lv, 1)
        R[c0:c1] = np.where(fin, Rv, 0)
        # exact re-decision of near-tie boundaries for the given FP64 lambda
        for i in np.nonzero(fin)[0]:
            g = i + c0
            tol = 1e-6 * max(1.0, abs(Nv[i]))
            near = False
            for kk in (int(L[g]) - 1, int(L[g]), int(R[g]), int(R[g]) + 1):
                if hk[0] <= kk <= hk[-1]:
                    if abs(float(cover_value(hk, hs, kk)) + lm[i] * kk - thr[i]) < tol:
                        near = True
            if not near:
                continue
            lamf = float(lm[i])
            ks = int(hk[istar[i]])
            th = Fraction(int(hs[istar[i]])) + Fraction(lamf) * ks - T
            l = int(L[g])
            while l < ks and _f_exact(hk, hs, l, lamf) < th:
                l += 1
            while l - 1 >= hk[0] and _f_exact(hk, hs, l - 1, lamf) >= th:
                l -= 1
            r = int(R[g])
            while r > ks and _f_exact(hk, hs, r, lamf) < th:
                r -= 1
            while r + 1 <= hk[-1] and _f_exact(hk, hs, r + 1, lamf) >= th:
                r += 1
            L[g], R[g] = l, r
    return kl, N, L, R


def windows_bruteforce(hk, hs, T: int, lam: float):
    """Exact (k_lambda, N, l, r) for one FP64 lambda by scanning every integer
    k of [k_0, k_last] in rational arithmetic (small degrees only)."""
    lamf = Fraction(lam)
    ks = list(range(int(hk[0]), int(hk[-1]) + 1))
    f = [cover_value(hk, hs, k) + lamf * k for k in ks]
    Nex = max(f)
    kstar = ks[f.index(Nex)]
    th = Nex - T
    i = ks.index(kstar)
    l = i
    while l - 1 >= 0 and f[l - 1] >= th:
        l -= 1
    r = i
    while r + 1 < len(ks) and f[r + 1] >= th:
        r += 1
    return kstar, Nex, ks[l], ks[r]


# ----------------------------------------------------------------------------
# extended double-double evaluation (C)
# ----------------------------------------------------------------------------

_lib = None


def _load():
    global _lib
    if _lib is None:
        from . import build as _b
        path = _b.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        lib.oracle_horner.argtypes = [I, P, P, P, P, P, I, P, P, P, P, P, P, P]
        lib.oracle_horner.restype = None
        lib.oracle_window_sum.argtypes = [I, P, P, P, P, P, P, I, P, P, P, P, P, P, P, P]
        lib.oracle_window_sum.restype = None
        lib.oracle_window_sum_fp64.argtypes = [I, P, P, P, P, I, P, P, P, P, P, P]
        lib.oracle_window_sum_fp64.restype = None
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class ExtValues:
    """Extended double-double results: value_j = ((re_hi+re_lo) + i(im_hi+im_lo)) 2^e_j."""

    def __init__(self, out4: np.ndarray, e: np.ndarray):
        self.re_hi, self.re_lo = out4[:, 0], out4[:, 1]
        self.im_hi, self.im_lo = out4[:, 2], out4[:, 3]
        self.e = e

    def fraction(self, j: int) -> Tuple[Fraction, Fraction]:
        sc = Fraction(2) ** int(self.e[j])
        return ((Fraction(float(self.re_hi[j])) + Fraction(float(self.re_lo[j]))) * sc,
                (Fraction(float(self.im_hi[j])) + Fraction(float(self.im_lo[j]))) * sc)


def horner_ref(coef, zre, zim=None, coef_lo=None):
    """P(z) over every term (ext double-double), S(z) = sum|a_k||z|^k as
    (mantissa, exponent), and log2 max_k |a_k z^k|."""
    lib = _load()
    are = _c(coef.re, np.float64)
    aim = _c(coef.im, np.float64)
    ae = _c(coef.e2, np.int64)
    are_lo = _c(coef_lo[0], np.float64) if coef_lo is not None else None
    aim_lo = _c(coef_lo[1], np.float64) if coef_lo is not None and coef_lo[1] is not None else None
    zre = _c(zre, np.float64)
    zim = _c(zim, np.float64)
    n = zre.shape[0]
    out = np.zeros((n, 4))
    oute = np.zeros(n, dtype=np.int64)
    Sm = np.zeros(n)
    Se = np.zeros(n, dtype=np.int64)
    lm = np.zeros(n)
    lib.oracle_horner(are.shape[0], _ptr(are), _ptr(aim), _ptr(are_lo), _ptr(aim_lo), _ptr(ae), n,
                      _ptr(zre), _ptr(zim), _ptr(out), _ptr(oute), _ptr(Sm), _ptr(Se), _ptr(lm))
    return ExtValues(out, oute), (Sm, Se), lm


def window_sum(coef, good: Optional[np.ndarray], zre, zim, lo, hi, coef_lo=None, with_S: bool = False):
    """sum over k in [lo_j, hi_j] with good[k] of a_k z_j^k (ext double-double);
    with_S also returns the window's sum of |a_k||z_j|^k as (mantissa, exponent)."""
    lib = _load()
    are = _c(coef.re, np.float64)
    aim = _c(coef.im, np.float64)
    ae = _c(coef.e2, np.int64)
    are_lo = _c(coef_lo[0], np.float64) if coef_lo is not None else None
    aim_lo = _c(coef_lo[1], np.float64) if coef_lo is not None and coef_lo[1] is not None else None
    g = _c(good, np.uint8)
    zre = _c(zre, np.float64)
    zim = _c(zim, np.float64)
    lo = _c(lo, np.int64)
    hi = _c(hi, np.int64)
    n = zre.shape[0]
    out = np.zeros((n, 4))
    oute = np.zeros(n, dtype=np.int64)
    Sm = np.zeros(n) if with_S else None
    Se = np.zeros(n, dtype=np.int64) if with_S else None
    lib.oracle_window_sum(are.shape[0], _ptr(are), _ptr(aim), _ptr(are_lo), _ptr(aim_lo), _ptr(ae),
                          _ptr(g), n, _ptr(zre), _ptr(zim), _ptr(lo), _ptr(hi), _ptr(out), _ptr(oute),
                          _ptr(Sm), _ptr(Se))
    if with_S:
        return ExtValues(out, oute), (Sm, Se)
    return ExtValues(out, oute)


def window_sum_fp64(coef, good: Optional[np.ndarray], zre, zim, lo, hi):
    """The same window sum with the Horner steps in plain FP64 (and a 64-bit
    exponent), z^lo in double-double: Algorithm A_p as a CPU program in hardware
    floats, for timing.  Its error is that of FP64 Horner over the window."""
    lib = _load()
    are = _c(coef.re, np.float64)
    aim = _c(coef.im, np.float64)
    ae = _c(coef.e2, np.int64)
    g = _c(good, np.uint8)
    zre = _c(zre, np.float64)
    zim = _c(zim, np.float64)
    lo = _c(lo, np.int64)
    hi = _c(hi, np.int64)
    n = zre.shape[0]
    out = np.zeros((n, 4))
    oute = np.zeros(n, dtype=np.int64)
    lib.oracle_window_sum_fp64(are.shape[0], _ptr(are), _ptr(aim), _ptr(ae), _ptr(g), n, _ptr(zre), _ptr(zim),
                               _ptr(lo), _ptr(hi), _ptr(out), _ptr(oute))
    return ExtValues(out, oute)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Number of OpenMP threads the C part uses from now on."""
    _load().oracle_set_threads(int(n))


# ----------------------------------------------------------------------------
# Algorithm A_p end to end
# ----------------------------------------------------------------------------

class Preconditioned:
    """Output of the preconditioning part of Algorithm A_p (§5.1)."""

    def __init__(self, coef, p: int):
        self.coef = coef
        self.p = p
        self.s = scale(coef.re, coef.im, coef.e2)
        nz = np.nonzero(self.s != NEG_INF)[0]
        if nz.size == 0:
            raise ValueError("zero polynomial")
        self.v = int(nz[0])   # valuation: first nonzero index
        self.d = int(nz[-1])  # degree: last nonzero index
        self.T = offset_T(p, self.d)
        self.hk, self.hs = concave_cover(self.s)
        self.good = good_mask(self.s, self.hk, self.hs, self.T)


def precondition(coef, p: int) -> Preconditioned:
    return Preconditioned(coef, p)


def fpe_eval_fp64(pre: Preconditioned, zre, zim=None):
    """Algorithm A_p evaluation with the window sums in plain FP64 (window_sum_fp64)."""
    lam = log2_abs(np.asarray(zre, dtype=np.float64), None if zim is None else np.asarray(zim, dtype=np.float64))
    kl, N, L, R = windows(pre.hk, pre.hs, pre.T, lam)
    zero = ~np.isfinite(lam)
    L2, R2 = L.copy(), R.copy()
    L2[zero] = 0
    R2[zero] = 0
    return window_sum_fp64(pre.coef, pre.good, zre, zim, L2, R2), (kl, N, L, R)


def fpe_eval(pre: Preconditioned, zre, zim=None, with_S: bool = False):
    """Algorithm A_p evaluation (§5.2): returns (values, (k_lambda, N, l, r)).
    At z = 0 the value is a_0 (§4.2: P(0) = a_0 is immediately available)."""
    lam = log2_abs(np.asarray(zre, dtype=np.float64), None if zim is None else np.asarray(zim, dtype=np.float64))
    kl, N, L, R = windows(pre.hk, pre.hs, pre.T, lam)
    zero = ~np.isfinite(lam)
    L2 = L.copy()
    R2 = R.copy()
    L2[zero] = 0
    R2[zero] = 0  # window {0}: P(0) = a_0 (0 when a_0 = 0)
    vals = window_sum(pre.coef, pre.good, zre, zim, L2, R2, with_S=with_S)
    return vals, (kl, N, L, R)
