"""Seeded synthetic inputs for fast polynomial evaluation (FPE) workloads.

This module only draws random numbers and lays out input arrays.  It holds no
part of the evaluation method (no scales, covers, windows or sums), so both
the CPU oracle and the CUDA path may take their inputs from here.

Coefficients are returned as ``Coeffs(re, im, e2)`` meaning
``a_k = (re[k] + i*im[k]) * 2**e2[k]``; ``im`` is ``None`` for a real
polynomial and ``e2`` is ``None`` when every exponent is zero.  Points are
returned as ``Points(re, im)`` with ``im`` ``None`` for real points.

Every generator takes an explicit seed and draws with
``numpy.random.default_rng(seed)`` (PCG64) in the order documented on it.

Workload shapes (the paper evaluates on synthetic families only, §8.3):
  * ``unit_square_complex``: d=1000, a_k = x + iy, x, y iid U[-1, 1], 10^4
    sphere-uniform points.
  * ``unit_disk_complex``: d=2^20, a_k uniform in the unit disk, 2^20
    sphere-uniform points (the headline workload).
  * ``inverse_factorial``: a_k = 1/k!, d=10^5, real points U[-50, 50].
  * ``mandelbrot``: hyperbolic-centre polynomial p_{n+1} = p_n^2 + c, p_0 = c.
  * ``sparse_real``: d=2^22, 1% of a_k nonzero U[-1, 1].
  * ``batched_lognormal``: 4096 polynomials with log-uniform degree in
    [16, 2^16] and log2|a_k| = s*k + N(0, 4).
  * ``half_circle``: the family sum 2^sqrt((n+1)(d+1-n)) z^n (eq. halfcirclepoly).
  * Chebyshev T_d monomial coefficients, geometric series, z^d - 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np


@dataclass
class Coeffs:
    re: np.ndarray
    im: Optional[np.ndarray] = None
    e2: Optional[np.ndarray] = None

    @property
    def n_coef(self) -> int:
        return int(self.re.shape[0])

    def is_real(self) -> bool:
        return self.im is None


@dataclass
class Points:
    re: np.ndarray
    im: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.re.shape[0])

    def is_real(self) -> bool:
        return self.im is None


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------

def sphere_points(n: int, rng: np.random.Generator) -> Points:
    """Uniform on the Riemann sphere: cos(theta) ~ U[-1, 1], phi ~ U[0, 2pi),
    z = tan(theta/2) e^{i phi} = sqrt((1-c)/(1+c)) e^{i phi}.
    Draw order: all cos(theta) values, then all phi values."""
    c = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    with np.errstate(divide="ignore"):
        r = np.sqrt((1.0 - c) / (1.0 + c))
    return Points(np.ascontiguousarray(r * np.cos(phi)), np.ascontiguousarray(r * np.sin(phi)))


def disk_points(n: int, rng: np.random.Generator) -> Points:
    """Uniform on the unit disk: r = sqrt(U), phi ~ U[0, 2pi)."""
    r = np.sqrt(rng.uniform(0.0, 1.0, n))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    return Points(r * np.cos(phi), r * np.sin(phi))


def real_line_points(n: int, lo: float, hi: float, rng: np.random.Generator) -> Points:
    return Points(rng.uniform(lo, hi, n))


def real_circle_points(n: int, rng: np.random.Generator) -> Points:
    """Uniform on the real projective line R u {inf} (stereographic):
    x = tan(t/2) with t ~ U(-pi, pi)."""
    t = rng.uniform(-math.pi, math.pi, n)
    return Points(np.tan(t / 2.0))


# ----------------------------------------------------------------------------
# coefficient families
# ----------------------------------------------------------------------------

def unit_square_complex(d: int, rng: np.random.Generator) -> Coeffs:
    """a_k = x + iy with x, y iid U[-1, 1]; one (d+1, 2) draw, column 0 = x."""
    xy = rng.uniform(-1.0, 1.0, (d + 1, 2))
    return Coeffs(np.ascontiguousarray(xy[:, 0]), np.ascontiguousarray(xy[:, 1]))


def unit_disk_complex(d: int, rng: np.random.Generator) -> Coeffs:
    """a_k uniform in the unit disk: modulus sqrt(U), phase 2*pi*U'."""
    r = np.sqrt(rng.uniform(0.0, 1.0, d + 1))
    ph = rng.uniform(0.0, 2.0 * math.pi, d + 1)
    return Coeffs(r * np.cos(ph), r * np.sin(ph))


def _ext_normalise(m: np.ndarray, e: np.ndarray):
    """Return (mantissa, exponent) with |mantissa| in [0.5, 1) or 0."""
    fm, fe = np.frexp(m)
    return fm, (e + fe).astype(np.int64)


def inverse_factorial(d: int) -> Coeffs:
    """a_k = 1/k! as an extended-exponent FP64 sequence built by the
    recurrence a_k = a_{k-1}/k, rounding once per step (plain FP64 underflows
    past k ~ 170, so the exponent is carried separately)."""
    m = np.empty(d + 1)
    e = np.zeros(d + 1, dtype=np.int64)
    cur_m, cur_e = 1.0, 0
    m[0] = 1.0
    for k in range(1, d + 1):
        cur_m = cur_m / k
        fm, fe = math.frexp(cur_m)
        cur_m, cur_e = fm, cur_e + fe
        m[k], e[k] = cur_m, cur_e
    return Coeffs(m, None, e)


def mandelbrot(n: int) -> Coeffs:
    """Coefficients of p_n with p_0 = c, p_{k+1} = p_k^2 + c (degree 2^n),
    as extended-exponent FP64 (the integer coefficients exceed the FP64
    range for n >= 11).  Each squaring is a direct convolution: output k sums
    m_j m_{k-j} 2^{e_j + e_{k-j} - G_k} with G_k the largest exponent of its
    terms; all terms are positive, so this keeps full relative precision.
    The convolution is O(d^2), practical up to n ~ 14."""
    m = np.array([0.0, 0.5])          # p_0 = c  ->  a_1 = 1 = 0.5 * 2^1
    e = np.array([0, 1], dtype=np.int64)
    for _ in range(n):
        L = m.shape[0]
        dd = 2 * (L - 1)
        out_m = np.zeros(dd + 1)
        out_e = np.zeros(dd + 1, dtype=np.int64)
        nzi = np.nonzero(m)[0]
        for k in range(dd + 1):
            j = nzi[(nzi <= k) & (nzi >= k - (L - 1))]
            j = j[m[k - j] != 0.0]
            if j.size == 0:
                continue
            ex = e[j] + e[k - j]
            G = int(ex.max())
            s = float(np.sum(m[j] * m[k - j] * np.exp2((ex - G).astype(np.float64))))
            fm, fe = math.frexp(s)
            out_m[k], out_e[k] = fm, G + fe
        # + c
        if out_m[1] == 0.0:
            out_m[1], out_e[1] = 0.5, 1
        else:
            s = out_m[1] + math.ldexp(1.0, -int(out_e[1]))
            fm, fe = math.frexp(s)
            out_m[1], out_e[1] = fm, int(out_e[1]) + fe
        m, e = out_m, out_e
    return Coeffs(m, None, e)


def mandelbrot_fast(n: int) -> Coeffs:
    """mandelbrot(n) by the C generator (mandelbrot_gen.c: the same convolution,
    each output summed over the terms within 2^-128 of its largest, OpenMP),
    practical up to n = 20; compiled with gcc on first use into a build
    folder beside this file."""
    import ctypes
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "mandelbrot_gen.c")
    out_dir = os.path.join(here, "_build")
    lib = os.path.join(out_dir, "mandelbrot_gen.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, lib)
    L = ctypes.CDLL(lib)
    L.mandel_coeffs.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.mandel_coeffs.restype = ctypes.c_int
    N = (1 << n) + 1
    m = np.zeros(N)
    e = np.zeros(N, dtype=np.int64)
    if L.mandel_coeffs(int(n), m.ctypes.data, e.ctypes.data) != 0:
        raise MemoryError("mandel_coeffs")
    return Coeffs(m, None, e)


def sparse_real(d: int, density: float, rng: np.random.Generator) -> Coeffs:
    """Bernoulli(density) mask then values U[-1, 1]; a_d forced nonzero.
    Draw order: mask uniforms (d+1), then values (d+1)."""
    mask = rng.uniform(0.0, 1.0, d + 1) < density
    vals = rng.uniform(-1.0, 1.0, d + 1)
    mask[d] = True
    if vals[d] == 0.0:
        vals[d] = 0.5
    return Coeffs(np.where(mask, vals, 0.0))


def lognormal_profile(d: int, slope: float, rng: np.random.Generator) -> Coeffs:
    """log2|a_k| = slope*k + N(0, 4) (variance 4), phase U[0, 2pi).
    Draw order: normals (d+1), phases (d+1)."""
    g = rng.normal(0.0, 2.0, d + 1)
    ph = rng.uniform(0.0, 2.0 * math.pi, d + 1)
    lg = slope * np.arange(d + 1) + g
    mod = np.exp2(lg)
    return Coeffs(mod * np.cos(ph), mod * np.sin(ph))


def half_circle(d: int, complex_phase: bool = False, rng: Optional[np.random.Generator] = None) -> Coeffs:
    """a_n = 2^sqrt((n+1)(d+1-n)) (eq. halfcirclepoly); with complex_phase a
    uniform random phase multiplies each coefficient."""
    n = np.arange(d + 1, dtype=np.float64)
    lg = np.sqrt((n + 1.0) * (d + 1.0 - n))
    ge = np.floor(lg).astype(np.int64)
    mant = np.exp2(lg - ge)
    m, e = _ext_normalise(mant, ge)
    if complex_phase:
        assert rng is not None
        ph = rng.uniform(0.0, 2.0 * math.pi, d + 1)
        return Coeffs(m * np.cos(ph), m * np.sin(ph), e)
    return Coeffs(m, None, e)


def chebyshev_T(d: int) -> Coeffs:
    """Monomial coefficients of the Chebyshev polynomial T_d, built from the
    three-term recurrence in exact integers and rounded once to an
    extended-exponent FP64 value."""
    t0 = [1]
    t1 = [0, 1]
    if d == 0:
        ints = t0
    else:
        for _ in range(d - 1):
            nxt = [0] * (len(t1) + 1)
            for i, c in enumerate(t1):
                nxt[i + 1] += 2 * c
            for i, c in enumerate(t0):
                nxt[i] -= c
            t0, t1 = t1, nxt
        ints = t1
    m = np.zeros(len(ints))
    e = np.zeros(len(ints), dtype=np.int64)
    for k, c in enumerate(ints):
        if c == 0:
            continue
        sh = max(0, abs(c).bit_length() - 60)
        fm, fe = math.frexp(float(c >> sh) if c > 0 else -float((-c) >> sh))
        # c >> sh keeps >= 53 leading bits; correct rounding of the tail is
        # not needed for a test input (both sides read the same value)
        m[k], e[k] = fm, fe + sh
    return Coeffs(m, None, e)


def geometric(d: int) -> Coeffs:
    """All coefficients 1: sum z^k = (z^{d+1} - 1)/(z - 1)."""
    return Coeffs(np.ones(d + 1))


def power_minus_one(d: int) -> Coeffs:
    """z^d - 1."""
    c = np.zeros(d + 1)
    c[0] = -1.0
    c[d] = 1.0
    return Coeffs(c)


def worked_example_scales() -> List[int]:
    """s(a_k) of the degree-10 example of §4.1 (A simple example detailed)."""
    return [-2, 6, -3, 16, 14, -4, 27, 16, 30, 30, 18]


def worked_example_coeffs(rng: np.random.Generator) -> Coeffs:
    """Coefficients whose moduli are exactly the powers of two printed in the
    §4.1 table (|a_k| = 2^{s_k - 1}), with random phases (the example states
    the phases are irrelevant)."""
    s = np.array(worked_example_scales(), dtype=np.int64)
    ph = rng.uniform(0.0, 2.0 * math.pi, s.shape[0])
    return Coeffs(np.cos(ph), np.sin(ph), s - 1)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    coeffs: Coeffs
    points: Points
    p: int


def unit_square_d1000(n_points: int = 10_000) -> Workload:
    """d=1000, a_k = x+iy with x, y iid U[-1,1] (seed 0), 10^4 sphere points."""
    rng = np.random.default_rng(0)
    c = unit_square_complex(1000, rng)
    z = sphere_points(n_points, rng)
    return Workload("unit_square_d1000", c, z, 53)


def unit_disk_d2pow20(n_points: int = 1 << 20, d: int = 1 << 20) -> Workload:
    """d=2^20, a_k uniform in the unit disk (seed 1), 2^20 sphere points."""
    rng = np.random.default_rng(1)
    c = unit_disk_complex(d, rng)
    z = sphere_points(n_points, rng)
    return Workload(f"unit_disk_d{d}", c, z, 53)


def inverse_factorial_d1e5(n_points: int = 1 << 20, d: int = 100_000) -> Workload:
    """a_k = 1/k!, d=10^5; real points U[-50, 50] (seed 2)."""
    rng = np.random.default_rng(2)
    return Workload("inverse_factorial", inverse_factorial(d), real_line_points(n_points, -50.0, 50.0, rng), 53)


def mandelbrot_real(n: int, n_points: int = 1 << 20) -> Workload:
    """Hyperbolic-centre polynomial p_n (degree 2^n); real points U[-2, 0.25] (seed 2).
    n > 12 uses the C generator (mandelbrot_fast)."""
    rng = np.random.default_rng(2)
    coef = mandelbrot(n) if n <= 12 else mandelbrot_fast(n)
    return Workload(f"mandelbrot_n{n}", coef, real_line_points(n_points, -2.0, 0.25, rng), 53)


def sparse_d2pow22(n_points: int = 1 << 20, d: int = 1 << 22) -> Workload:
    """d=2^22, 1% nonzero U[-1,1] real coefficients; sphere points (seed 2)."""
    rng = np.random.default_rng(2)
    c = sparse_real(d, 0.01, rng)
    return Workload("sparse_real", c, sphere_points(n_points, rng), 53)


def batched_lognormal(n_poly: int = 4096, pts_per_poly: int = 256, seed: int = 3,
                      dmin: int = 16, dmax: int = 1 << 16) -> List[Workload]:
    """n_poly polynomials: d = round(exp(U[ln dmin, ln dmax])), slope s ~
    U[-0.01, 0.01], log2|a_k| = s k + N(0,4), pts_per_poly sphere points each.
    Draw order per polynomial: degree, slope, coefficients, points."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_poly):
        d = int(round(math.exp(rng.uniform(math.log(dmin), math.log(dmax)))))
        slope = rng.uniform(-0.01, 0.01)
        c = lognormal_profile(d, slope, rng)
        z = sphere_points(pts_per_poly, rng)
        out.append(Workload(f"batched_{i}", c, z, 53))
    return out


def differentiation_d2pow18(n_points: int = 1 << 20, d: int = 1 << 18, seed: int = 4):
    """d=2^18 unit-disk coefficients a_true, observed a = a_true + 1e-3 CN(0,1),
    sphere points.  Returns (workload with a, a_true, noise for targets).
    Draw order: a_true, coefficient noise (d+1, 2), points, target noise (n, 2)."""
    rng = np.random.default_rng(seed)
    a_true = unit_disk_complex(d, rng)
    nz = rng.normal(0.0, 1.0, (d + 1, 2)) * 1e-3
    a = Coeffs(a_true.re + nz[:, 0], a_true.im + nz[:, 1])
    z = sphere_points(n_points, rng)
    tn = rng.normal(0.0, 1.0, (n_points, 2)) * 1e-3
    return Workload("differentiation", a, z, 53), a_true, tn
