"""Fixed-point bookkeeping of the window kernels (fpe_device.cuh), compiled
as host code, against exact rational arithmetic: exact conversion of
double-double values, addition, the Newton reciprocal 1/m used for the
bottom-up multiplier and its powers, and the conversion of z^n to the output
format."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U64x4 = ctypes.c_uint64 * 4
I32x2 = ctypes.c_int * 2


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("xint") / "xint_host.so")
    cmd = [nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2211_06320_gb300", "csrc"),
           os.path.join(ROOT, "tests", "native", "xint_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    D, LL, P = ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
    L.t_recip.argtypes = [D, D, P, P, P]
    L.t_from_dd2.argtypes = [D, D, D, D, LL, P, P, P]
    L.t_add.argtypes = [D, D, LL, D, D, LL, P, P, P]
    L.t_pow_out.argtypes = [D, D, LL, P, P, P]
    return L


def _val(o, s, e):
    x = int(o[0]) | (int(o[1]) << 64)
    y = int(o[2]) | (int(o[3]) << 64)
    sc = Fraction(2) ** (int(e.value) - 126)
    return Fraction(-x if s[0] else x) * sc, Fraction(-y if s[1] else y) * sc


def _call(fn, *args):
    o, s, e = U64x4(), I32x2(), ctypes.c_longlong()
    fn(*args, o, s, ctypes.byref(e))
    return _val(o, s, e)


def _abs2(re, im):
    return re * re + im * im


def test_from_dd2_and_add_exact(lib):
    rng = np.random.default_rng(5)
    for _ in range(300):
        rh, ih = rng.normal() * 2.0 ** rng.integers(-40, 40), rng.normal() * 2.0 ** rng.integers(-40, 40)
        if rng.random() < 0.2:
            ih = 0.0
        rl = float(np.spacing(rh)) * rng.uniform(-0.5, 0.5) if rh else 0.0
        il = float(np.spacing(ih)) * rng.uniform(-0.5, 0.5) if ih else 0.0
        e0 = int(rng.integers(-100, 100))
        gr, gi = _call(lib.t_from_dd2, rh, rl, ih, il, e0)
        sc = Fraction(2) ** e0
        wr, wi = (Fraction(rh) + Fraction(rl)) * sc, (Fraction(ih) + Fraction(il)) * sc
        big = max(abs(wr), abs(wi))
        assert abs(gr - wr) <= big * Fraction(1, 2 ** 120) and abs(gi - wi) <= big * Fraction(1, 2 ** 120)
        ar, ai, br, bi = rng.normal(size=4)
        ae, be = int(rng.integers(-60, 60)), int(rng.integers(-60, 60))
        gr, gi = _call(lib.t_add, ar, ai, ae, br, bi, be)
        wr = Fraction(ar) * Fraction(2) ** ae + Fraction(br) * Fraction(2) ** be
        wi = Fraction(ai) * Fraction(2) ** ae + Fraction(bi) * Fraction(2) ** be
        ref = max(abs(Fraction(ar)), abs(Fraction(ai))) * Fraction(2) ** ae + \
            max(abs(Fraction(br)), abs(Fraction(bi))) * Fraction(2) ** be
        assert abs(gr - wr) <= ref * Fraction(1, 2 ** 120) and abs(gi - wi) <= ref * Fraction(1, 2 ** 120)


def test_recip_newton(lib):
    rng = np.random.default_rng(6)
    cases = [(0.5, 0.0), (-0.75, 0.0), (0.0, 0.5), (0.999, -0.999), (0.5, 0.5)]
    for _ in range(300):
        t = rng.uniform(0, 2 * np.pi)
        r = rng.uniform(0.5, 1.0)
        mr, mi = r * np.cos(t), r * np.sin(t)
        mx = max(abs(mr), abs(mi))
        k = np.floor(np.log2(mx)) + 1  # scale so max(|mr|, |mi|) lies in [0.5, 1)
        cases.append((mr * 2.0 ** -k, mi * 2.0 ** -k))
    for mr, mi in cases:
        gr, gi = _call(lib.t_recip, mr, mi)
        M = (Fraction(mr), Fraction(mi))
        n2 = _abs2(*M)
        wr, wi = M[0] / n2, -M[1] / n2
        err2 = _abs2(gr - wr, gi - wi)
        assert err2 <= _abs2(wr, wi) * Fraction(1, 2 ** 196), (mr, mi)  # relative error below 2^-98


def test_pow_to_output(lib):
    rng = np.random.default_rng(7)
    for _ in range(60):
        zr, zi = rng.normal() * 2.0 ** rng.integers(-4, 4), rng.normal()
        n = int(rng.integers(0, 300))
        re, im, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        lib.t_pow_out(zr, zi, n, ctypes.byref(re), ctypes.byref(im), ctypes.byref(e))
        assert 0.5 <= max(abs(re.value), abs(im.value)) < 1.0
        w = (Fraction(zr), Fraction(zi))
        acc = (Fraction(1), Fraction(0))
        for _ in range(n):
            acc = (acc[0] * w[0] - acc[1] * w[1], acc[0] * w[1] + acc[1] * w[0])
        sc = Fraction(2) ** int(e.value)
        got = (Fraction(re.value) * sc, Fraction(im.value) * sc)
        err2 = _abs2(got[0] - acc[0], got[1] - acc[1])
        assert err2 <= _abs2(*acc) * Fraction(1, 2 ** 100)  # 53-bit output: relative error below 2^-50
