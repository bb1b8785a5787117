"""Integer arithmetic of the tensor-core window sums (fpe_tc_arith.cuh),
compiled as host code, against exact integers and rationals:

- the balanced base-128 digits of a 69-bit operand and their bf16 encoding
  reconstruct the operand exactly, within the stated digit ranges;
- the join of ten fp32 accumulators is the exact sum_t v_t 128^(9 - t);
- one MMA output row (64 digit products per pair, pairs s + s' <= 9): every
  fp32 accumulator is the exact integer sum and stays below 2^22 even for
  digits at their extremes, the join equals the kept pairs' sum, and the
  dropped pairs stay below 2^-66 of the product scale per product;
- the 64-bit-mantissa complex product and sum (xh) are within 2^-60 of the
  exact values relative to their operands, the conversion from 128 bits
  within 2^-63.
"""
import ctypes
import os
import random
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U64 = ctypes.c_uint64
K = 64  # contraction length of one MMA row (32 terms x re, im)
SL = 10


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tcarith") / "tc_arith_host.so")
    cmd = [nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2211_06320_gb300", "csrc"),
           os.path.join(ROOT, "tests", "native", "tc_arith_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.t_digits.argtypes = [P, ctypes.c_uint, P, P]
    L.t_join.argtypes = [P, P, P]
    L.t_row.argtypes = [P, P, P, P, P, P, P]
    for f in (L.t_xh_mul, L.t_xh_add):
        f.argtypes = [P, P, ctypes.c_longlong, P, P, ctypes.c_longlong, P, P, P]
    L.t_xh_from128.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_longlong, P, P, P]
    return L


def _words(v):
    return (U64 * 2)(v & (2**64 - 1), v >> 64)


def _bf16_to_int(h):
    f = np.array([int(x) << 16 for x in h], dtype=np.uint32).view(np.float32)
    assert np.all(f == np.round(f))
    return [int(x) for x in f]


def _digits(lib, F, neg):
    lo = (ctypes.c_ushort * SL)()
    hi = (ctypes.c_ushort * SL)()
    lib.t_digits(_words(F), neg, lo, hi)
    assert list(lo) == list(hi)
    return _bf16_to_int(lo)


def _extreme_operands(rng):
    """69-bit operands whose balanced digits sit at +-64 (the largest digit products)."""
    out = []
    for _ in range(8):
        ds = [64] + [rng.choice((-64, 63)) for _ in range(SL - 1)]
        v = 0
        for d in ds:
            v = v * 128 + d
        if 0 <= v < 2**69:
            out.append(v)
    out.append(2**69 - 1)
    return out


def test_digits_reconstruct(lib):
    rng = random.Random(1)
    cases = [0, 1, 63, 64, 127, 128, 2**63, 2**69 - 1, 2**69 - 2**62] + _extreme_operands(rng)
    cases += [rng.getrandbits(69) for _ in range(3000)] + [rng.getrandbits(rng.randint(1, 69)) for _ in range(1000)]
    for F in cases:
        for neg in (0, 1):
            d = _digits(lib, F, neg)
            sgn = -1 if neg else 1
            assert sum(x * 128 ** (SL - 1 - j) for j, x in enumerate(d)) == sgn * F, (F, neg, d)
            u = [sgn * x for x in d]
            assert 0 <= u[0] <= 64
            assert all(-64 <= x <= 63 for x in u[1:])


def test_join_exact(lib):
    rng = random.Random(2)
    mag = (U64 * 2)()
    neg = ctypes.c_int()
    lim = 2**22
    vecs = [[lim - 1] * SL, [-lim] * SL, [0] * SL, [1] + [0] * 9, [0] * 9 + [-1]]
    vecs += [[rng.randint(-lim, lim - 1) for _ in range(SL)] for _ in range(5000)]
    for v in vecs:
        lib.t_join((ctypes.c_float * SL)(*v), mag, ctypes.byref(neg))
        X = (mag[0] | (mag[1] << 64)) * (-1 if neg.value else 1)
        assert X == sum(x * 128 ** (SL - 1 - t) for t, x in enumerate(v)), v


def _row(lib, a, asg, z, zsg):
    A = (U64 * (2 * K))(*[w for v in a for w in (v & (2**64 - 1), v >> 64)])
    Z = (U64 * (2 * K))(*[w for v in z for w in (v & (2**64 - 1), v >> 64)])
    mag = (U64 * 2)()
    neg = ctypes.c_int()
    ex = (ctypes.c_longlong * (2 * SL))()
    lib.t_row(A, (ctypes.c_int * K)(*asg), Z, (ctypes.c_int * K)(*zsg), mag, ctypes.byref(neg), ex)
    X = (mag[0] | (mag[1] << 64)) * (-1 if neg.value else 1)
    return X, list(ex[:SL]), list(ex[SL:])


def _balanced(F):
    d = []
    for _ in range(SL):
        r = F % 128
        if r >= 64:
            r -= 128
        d.append(r)
        F = (F - r) // 128
    d.reverse()
    d[0] += F * 128 if F else 0
    return d


def test_mma_row_exact(lib):
    """Accumulators exact and below 2^22; join = kept pairs; dropped pairs tiny."""
    rng = random.Random(3)
    ext = _extreme_operands(rng)
    # the largest possible dropped-pair sum with |digits| <= 64, per product
    drop = sum((2 * SL - 1 - t) * 64 * 64 * Fraction(1, 128 ** (t - (SL - 1))) for t in range(SL, 2 * SL - 1))
    scale = Fraction(2**69 * 2**69, 128 ** (SL - 1))  # largest product in the join's units
    assert drop / scale < Fraction(1, 2**66)
    for trial in range(60):
        if trial == 0:  # every digit 63: every product +3969, the largest accumulators
            a = z = [sum(63 * 128**j for j in range(SL))] * K
            asg = zsg = [0] * K
        elif trial < 20:  # digits at their extremes
            a = [rng.choice(ext) for _ in range(K)]
            z = [rng.choice(ext) for _ in range(K)]
            asg = [rng.randint(0, 1)] * K
            zsg = [rng.randint(0, 1)] * K
        else:
            a = [rng.getrandbits(69) for _ in range(K)]
            z = [rng.getrandbits(rng.choice((69, 60, 40))) for _ in range(K)]
            asg = [rng.randint(0, 1) for _ in range(K)]
            zsg = [rng.randint(0, 1) for _ in range(K)]
        X, ex, acc = _row(lib, a, asg, z, zsg)
        assert acc == ex, "an fp32 accumulator was rounded"
        assert max(abs(v) for v in ex) < 2**22
        if trial == 0:
            assert ex[SL - 1] == SL * K * 63 * 63  # 2^21.3
        # kept pairs from Python's own balanced digits
        kept = 0
        for k in range(K):
            da = [(-x if asg[k] else x) for x in _balanced(a[k])]
            dz = [(-x if zsg[k] else x) for x in _balanced(z[k])]
            for s in range(SL):
                for s2 in range(SL - s):
                    kept += da[s] * dz[s2] * 128 ** (SL - 1 - s - s2)
        assert X == kept
        exact = Fraction(sum((-1) ** (asg[k] ^ zsg[k]) * a[k] * z[k] for k in range(K)), 128 ** (SL - 1))
        assert abs(exact - X) <= K * drop


def _xh(rng, zero_part=False):
    x = rng.getrandbits(64) | (1 << 63)
    y = rng.getrandbits(rng.choice((64, 50, 10))) if not zero_part else 0
    if rng.random() < 0.5:
        x, y = y, x
    return (U64 * 2)(x, y), (ctypes.c_int * 2)(rng.randint(0, 1), rng.randint(0, 1)), rng.randint(-200, 200)


def _exact(m, s, e):
    f = Fraction(2) ** (e - 63)
    return ((-1) ** s[0] * m[0] * f, (-1) ** s[1] * m[1] * f)


def _call_xh(fn, a, b):
    m = (U64 * 2)()
    s = (ctypes.c_int * 2)()
    e = ctypes.c_longlong()
    fn(a[0], a[1], a[2], b[0], b[1], b[2], m, s, ctypes.byref(e))
    assert max(m[0], m[1]) >= 2**63 or (m[0] == 0 and m[1] == 0)
    return _exact(m, s, e.value)


def test_xh_mul_add(lib):
    rng = random.Random(4)
    for _ in range(3000):
        a, b = _xh(rng, rng.random() < 0.1), _xh(rng, rng.random() < 0.1)
        ar, ai = _exact(*a)
        br, bi = _exact(*b)
        # product: two truncated high products, each halved: within 4 units of
        # 2^-62, i.e. 2^-60, of |a|max |b|max per component
        pr, pi = _call_xh(lib.t_xh_mul, a, b)
        bound = max(abs(ar), abs(ai)) * max(abs(br), abs(bi)) * Fraction(1, 2**60)
        assert abs(pr - (ar * br - ai * bi)) <= bound
        assert abs(pi - (ar * bi + ai * br)) <= bound
        # sum: the aligned and halved operands, within 2^-60 of the larger one's largest component
        sr, si = _call_xh(lib.t_xh_add, a, b)
        bound = max(abs(ar), abs(ai), abs(br), abs(bi)) * Fraction(1, 2**60)
        assert abs(sr - (ar + br)) <= bound
        assert abs(si - (ai + bi)) <= bound


def test_xh_from128(lib):
    rng = random.Random(5)
    m = (U64 * 2)()
    s = (ctypes.c_int * 2)()
    e = ctypes.c_longlong()
    for _ in range(2000):
        X = rng.getrandbits(rng.randint(1, 127))
        Y = rng.getrandbits(rng.randint(1, 127))
        sx, sy, e0 = rng.randint(0, 1), rng.randint(0, 1), rng.randint(-500, 500)
        lib.t_xh_from128(_words(X), sx, _words(Y), sy, e0, m, s, ctypes.byref(e))
        f = Fraction(2) ** (e0 - 126)
        vr, vi = (-1) ** sx * X * f, (-1) ** sy * Y * f
        gr, gi = _exact(m, s, e.value)
        bound = max(X, Y) * f * Fraction(1, 2**63)
        assert abs(gr - vr) <= bound and abs(gi - vi) <= bound
        assert abs(gr) <= abs(vr) and abs(gi) <= abs(vi)  # truncation toward zero
