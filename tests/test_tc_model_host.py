"""Error of the tensor-core window sums' arithmetic on adversarial tiles.

tests/native/tc_model_host.cu runs one tile through the same fixed-point
steps as the kernels (fpe_tc_arith.cuh and the xint helpers, compiled as
host code; the MMAs become exact integer dot products of the same digits).
Its value, sum over the tile's blocks of b_k z^k, must be within
2^-53.5 S of a 400-bit sum (S = sum |b_k| |z|^k over the same terms) -- the
bound the tensor path claims for tiles whose points lie within the planner's
tilt spread (31 |mu - c| <= 2) -- on:
- unit-disk coefficients with points at both edges of the allowed spread;
- the geometric series near z = 1 (every term aligned: truncation biases add);
- coefficients spread over 2^-60..1 inside the piece (per-block scales);
- several work items per tile, joined by one thread (<= 4 items) or eight.
"""
import ctypes
import math
import os
import random
import shutil
import subprocess

import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BOUND = 2.0 ** -53.5


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tcmodel") / "tc_model_host.so")
    cmd = [nvcc, "-x", "cu", "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2211_06320_gb300", "csrc"),
           os.path.join(ROOT, "tests", "native", "tc_model_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.t_tile.argtypes = [P, ctypes.c_longlong, ctypes.c_longlong, P, P, ctypes.c_int, ctypes.c_double,
                         ctypes.c_longlong, P, P, P]
    return L


def _run(lib, coef, mlo, nblk, pts, c, chunk):
    n = len(pts)
    b = (ctypes.c_double * (2 * len(coef)))(*[x for z in coef for x in (z.real, z.imag)])
    zr = (ctypes.c_double * n)(*[z.real for z in pts])
    zi = (ctypes.c_double * n)(*[z.imag for z in pts])
    ox = (ctypes.c_uint64 * (4 * n))()
    os_ = (ctypes.c_int * (2 * n))()
    oe = (ctypes.c_longlong * n)()
    lib.t_tile(b, mlo, nblk, zr, zi, n, c, chunk, ox, os_, oe)
    out = []
    with mpmath.workprec(400):  # the 128-bit result exactly (mpmath's default would round it to 53 bits)
        for p in range(n):
            X = ox[4 * p] | (ox[4 * p + 1] << 64)
            Y = ox[4 * p + 2] | (ox[4 * p + 3] << 64)
            out.append(mpmath.mpc(mpmath.ldexp((-1) ** os_[2 * p] * X, oe[p] - 126),
                                  mpmath.ldexp((-1) ** os_[2 * p + 1] * Y, oe[p] - 126)))
    return out


def _check(lib, coef, mlo, nblk, pts, c, chunk):
    assert len(coef) == 32 * nblk
    got = _run(lib, coef, mlo, nblk, pts, c, chunk)
    worst = 0.0
    with mpmath.workprec(400):
        for p, z in enumerate(pts):
            zm = mpmath.mpc(z.real, z.imag)
            k0 = 32 * mlo
            # Horner over the tile's terms, then z^k0
            h = mpmath.mpc(0)
            for b in reversed(coef):
                h = h * zm + mpmath.mpc(b.real, b.imag)
            val = h * zm ** k0
            az = abs(zm)
            S = mpmath.fsum(abs(mpmath.mpc(b.real, b.imag)) * az ** (k0 + i) for i, b in enumerate(coef))
            err = float(abs(got[p] - val) / S)
            worst = max(worst, err)
    assert worst <= BOUND, f"{worst:.3g} = 2^{math.log2(worst):.2f} S"
    return worst


def _points(rng, c, n, spread=2.0 / 31):
    """n points with log2|z| at c - spread, c + spread and in between, random arguments."""
    mus = [c - spread, c + spread] + [c + rng.uniform(-spread, spread) for _ in range(n - 2)]
    return [2.0 ** m * complex(math.cos(t), math.sin(t)) for m, t in ((m, rng.uniform(0, 2 * math.pi)) for m in mus)]


def _disk(rng, n):
    out = []
    for _ in range(n):
        r, t = math.sqrt(rng.random()), rng.uniform(0, 2 * math.pi)
        out.append(r * complex(math.cos(t), math.sin(t)))
    return out


def test_unit_disk_tilt_edges(lib):
    rng = random.Random(11)
    for c in (0.0, -0.004, 0.003):
        nblk = 24
        _check(lib, _disk(rng, 32 * nblk), 5, nblk, _points(rng, c, 6), c, 256)


def test_geometric_aligned(lib):
    rng = random.Random(12)
    nblk = 40
    coef = [1.0 + 0j] * (32 * nblk)
    pts = [2.0 ** rng.uniform(-2e-4, 2e-4) * complex(math.cos(t), math.sin(t))
           for t in [0.0] + [rng.uniform(-1e-3, 1e-3) for _ in range(3)]]
    _check(lib, coef, 0, nblk, pts, 0.0, 256)


def test_geometric_long_tilt_edges(lib):
    """The tightest case found: 8192 aligned unit terms (one full work item,
    32 Horner steps per lane group) at z = 1 and at both edges of the tilt
    spread: about 2^-56.7 S (random tiles: about 2^-59)."""
    nblk = 256
    pts = [1.0 + 0j, 2.0 ** (2.0 / 31), 2.0 ** (-2.0 / 31), 2.0 ** -1e-5 * complex(math.cos(1e-4), math.sin(1e-4))]
    _check(lib, [1.0 + 0j] * (32 * nblk), 0, nblk, pts, 0.0, 256)


def test_wide_coefficient_range(lib):
    rng = random.Random(13)
    nblk = 16
    coef = [2.0 ** -((7 * k) % 61) * complex(math.cos(t), math.sin(t))
            for k, t in enumerate(rng.uniform(0, 2 * math.pi) for _ in range(32 * nblk))]
    _check(lib, coef, 3, nblk, _points(rng, 0.001, 5), 0.001, 256)


@pytest.mark.parametrize("nblk,chunk", [(40, 16), (100, 16)])  # 3 items (one thread), 7 items (eight)
def test_several_items(lib, nblk, chunk):
    rng = random.Random(14 + nblk)
    _check(lib, _disk(rng, 32 * nblk), 2, nblk, _points(rng, 0.0, 4, spread=0.3 / 31), 0.0, chunk)
