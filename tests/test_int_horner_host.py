"""The integer-pipe Horner step of the accurate window sums (fpe_device.cuh),
compiled as host code, against exact rational arithmetic (Python fractions):
top-down Horner over random windows with wide coefficient exponents, zero
runs, and points whose components are close or far apart in magnitude
(the shared-exponent and split multipliers).  The error must stay below
n 2^-100 times sum |b_k||z|^k (the bound stated for FPE_ACCURATE)."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("inthorner") / "int_horner_host.so")
    cmd = [nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2211_06320_gb300", "csrc"),
           os.path.join(ROOT, "tests", "native", "int_horner_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.int_horner.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.int_horner.restype = ctypes.c_int
    return L


def _run(L, br, bi, zr, zi, cz, cc):
    out = np.zeros(4, np.uint64)
    sg = np.zeros(2, np.int32)
    G = np.zeros(1, np.int64)
    br = np.ascontiguousarray(br, np.float64)
    bi = np.ascontiguousarray(bi, np.float64)
    split = L.int_horner(br.ctypes.data, bi.ctypes.data, len(br), zr, zi, cz, cc, out.ctypes.data,
                         sg.ctypes.data, G.ctypes.data)
    xr = int(out[0]) | (int(out[1]) << 64)
    xi = int(out[2]) | (int(out[3]) << 64)
    sc = Fraction(2) ** int(G[0])
    return Fraction(-xr if sg[0] else xr) * sc, Fraction(-xi if sg[1] else xi) * sc, split


def _exact(br, bi, zr, zi, cz, cc):
    Zr, Zi = Fraction(zr), Fraction(zi) if cz else Fraction(0)
    hr, hi = Fraction(br[-1]), Fraction(bi[-1]) if cc else Fraction(0)
    for k in range(len(br) - 2, -1, -1):
        hr, hi = hr * Zr - hi * Zi + Fraction(br[k]), hr * Zi + hi * Zr + (Fraction(bi[k]) if cc else 0)
    return hr, hi


def _sum_abs(br, bi, zr, zi, cz, cc):
    z = abs(complex(zr, zi if cz else 0.0))
    S = Fraction(0)
    zk = Fraction(1)
    for k in range(len(br)):
        S += Fraction(abs(complex(br[k], bi[k] if cc else 0.0))) * zk
        zk *= Fraction(z)
    return S


def test_int_horner_exact(lib):
    rng = np.random.default_rng(20221111)
    seen_split = set()
    for trial in range(240):
        n = int(rng.integers(1, 90))
        cz, cc = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        kind = trial % 4
        if kind == 0:
            zr, zi = rng.normal(), rng.normal()
        elif kind == 1:  # components far apart: the split multiplier
            zr, zi = rng.normal(), rng.normal() * 2.0 ** int(rng.integers(-80, -5))
            if rng.random() < 0.5:
                zr, zi = zi, zr
        elif kind == 2:
            t = rng.uniform(0, 2 * np.pi)
            zr, zi = np.cos(t), np.sin(t)
        else:
            zr, zi = rng.normal() * 2.0 ** int(rng.integers(-8, 8)), rng.normal() * 2.0 ** int(rng.integers(-8, 8))
        br = rng.normal(size=n) * 2.0 ** rng.integers(-40, 40, size=n)
        bi = rng.normal(size=n) * 2.0 ** rng.integers(-40, 40, size=n)
        zero = rng.random(n) < 0.2
        br[zero] = 0.0
        bi[zero & (rng.random(n) < 0.5)] = 0.0
        if trial % 17 == 0:  # a zero prefix: the frame comes from a later coefficient
            br[1:] = 0.0
            bi[1:] = 0.0
            br[0] = 1.0
        gr, gi, split = _run(lib, br, bi, zr, zi, cz, cc)
        if cz:
            seen_split.add(split)
        er, ei = _exact(br, bi, zr, zi, cz, cc)
        err = max(abs(gr - er), abs(gi - ei))
        S = _sum_abs(br, bi, zr, zi, cz, cc)
        assert err <= Fraction(n, 2 ** 100) * S, (trial, float(err / S) if S else err)
    assert seen_split == {0, 1}
