"""The certified FP64 window sums (fpe_window.cuh), compiled as host code,
against exact sums in big-integer arithmetic.

The top-down pass returns h with sum_{k=lo}^{hi} b_k 2^rho(k) z^(k-lo) =
h 2^rho(lo), the bottom-up pass h with sum b_k 2^rho(k) z^(k-hi) = h 2^rho(hi)
(Alg. A_p's window sum on the rescaled coefficients of §8.2).  Each also
returns a certificate (E, S): the claim checked here is

    |h - exact| <= 2^-113 E   (2^-53 per unit of E, at the scale 2^60),
    2^-60 S <= sum of the terms' magnitudes,

the bottom-up pass allowing in addition L 2^-96 times that sum for its
double-double multipliers 1/z, z^-3, z^-4.  The exact sums follow the plain
definition (rho(k) = rho0_j + beta_j (k - k0_j) on piece j, and the powers of
z), not the passes' piece crossings, so a wrong rescaling, a wrong power or a
wrong multiplier fails the value check, and a rounding left out of E shows
on inputs whose rounding errors pile up (terms of one sign at z close to 1).
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = ctypes.c_void_p
I, LL, D = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
LOG2_PIECE = 4


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("wcert") / "window_cert_host.so")
    cmd = [nvcc, "-x", "cu", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2211_06320_gb300", "csrc"),
           os.path.join(ROOT, "tests", "native", "window_cert_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.wc_top.argtypes = [P, I, I, P, P, P, P, P, I, I, D, D, LL, LL, P, P, P]
    L.wc_rev.argtypes = [P, I, I, P, P, P, P, P, I, I, D, D, LL, LL, I, P, P, P]
    L.wc_top.restype = I
    L.wc_rev.restype = I
    L.wc_mags.argtypes = [D, D, P]
    L.wc_step_w.argtypes = [I, I, D, D, D, D, D, D, P]
    L.wc_step_w.restype = ctypes.c_float
    L.wc_step_v.argtypes = [I, I, D, D, D, D, D, D, D, D, P]
    L.wc_step_v.restype = ctypes.c_float
    return L


# ------------------------------------------------------------ exact arithmetic
# A dyadic rational m 2^e as (m, e); complex values as pairs of them.

def dy(x):
    m, e = math.frexp(float(x))
    return (int(m * 2 ** 53), e - 53)


def dadd(a, b):
    if a[0] == 0:
        return b
    if b[0] == 0:
        return a
    e = min(a[1], b[1])
    return ((a[0] << (a[1] - e)) + (b[0] << (b[1] - e)), e)


def dmul(a, b):
    return (a[0] * b[0], a[1] + b[1])


def dneg(a):
    return (-a[0], a[1])


def cmul(a, b):
    return (dadd(dmul(a[0], b[0]), dneg(dmul(a[1], b[1]))), dadd(dmul(a[0], b[1]), dmul(a[1], b[0])))


def cadd(a, b):
    return (dadd(a[0], b[0]), dadd(a[1], b[1]))


def cscale2(a, k):
    return ((a[0][0], a[0][1] + k), (a[1][0], a[1][1] + k))


def to_float(a):
    m, e = a
    if m == 0:
        return 0.0
    sh = m.bit_length() - 60
    if sh > 0:
        m >>= sh
        e += sh
    return math.ldexp(float(m), e)


def abs2_le(d, bound2_m, bound2_e):
    """|d|^2 <= bound2 (bound2 = m 2^e, exact)"""
    s = dadd(dmul(d[0], d[0]), dmul(d[1], d[1]))
    e = min(s[1], bound2_e)
    return (s[0] << (s[1] - e)) <= (bound2_m << (bound2_e - e))


# ------------------------------------------------------------ inputs

def make_pieces(n, rng, beta_c, jump=3):
    """pieces on [0, n): cuts at multiples of 2^LOG2_PIECE plus random ones"""
    cuts = set(range(0, n, 1 << LOG2_PIECE)) | set(rng.integers(1, n, n // 24).tolist())
    k0 = sorted(cuts)
    npc = len(k0)
    beta = (beta_c + rng.integers(-1, 2, npc) * (rng.uniform(size=npc) < 0.25)).astype(np.int32)
    delta = rng.integers(-jump, jump + 1, npc).astype(np.int32)
    k0 = np.array(k0 + [n], dtype=np.int32)
    delta[-1] = 0
    rho0 = np.zeros(npc, np.int64)
    rho0[0] = int(rng.integers(-5, 6))
    for j in range(npc - 1):
        rho0[j + 1] = rho0[j] + int(beta[j]) * int(k0[j + 1] - k0[j]) + int(delta[j])
    nblk = ((n - 1) >> LOG2_PIECE) + 2
    first = np.zeros(nblk, np.int32)
    j = 0
    for g in range(nblk):
        while j + 1 < npc and k0[j + 1] <= (g << LOG2_PIECE):
            j += 1
        first[g] = j
    return k0, beta, delta, rho0, first


def rho_of(k, k0, beta, rho0):
    j = int(np.searchsorted(k0, k, side="right")) - 1
    return int(rho0[j]) + int(beta[j]) * (k - int(k0[j]))


def run(lib, kind, b, cc, cz, pieces, zr, zi, lo, hi, blocks=1):
    k0, beta, delta, rho0, first = pieces
    out = np.zeros(2)
    rho = np.zeros(1, np.int64)
    es = np.zeros(2, np.float32)
    args = [b.ctypes.data, cc, cz, k0.ctypes.data, beta.ctypes.data, delta.ctypes.data, rho0.ctypes.data,
            first.ctypes.data, len(beta), LOG2_PIECE, zr, zi, lo, hi]
    if kind == "top":
        ok = lib.wc_top(*args, out.ctypes.data, rho.ctypes.data, es.ctypes.data)
    else:
        ok = lib.wc_rev(*args, blocks, out.ctypes.data, rho.ctypes.data, es.ctypes.data)
    return bool(ok), out, int(rho[0]), float(es[0]), float(es[1])


def coef(b, cc, k):
    return (dy(b[2 * k]), dy(b[2 * k + 1])) if cc else (dy(b[k]), (0, 0))


def check_top(lib, b, cc, cz, pieces, zr, zi, lo, hi):
    k0, beta, delta, rho0, _ = pieces
    ok, out, rho, E, S = run(lib, "top", b, cc, cz, pieces, zr, zi, lo, hi)
    assert rho == rho_of(lo, k0, beta, rho0)
    z = (dy(zr), dy(zi if cz else 0.0))
    acc, pw, absum = ((0, 0), (0, 0)), ((1, 0), (0, 0)), 0.0
    r_lo = rho_of(lo, k0, beta, rho0)
    zabs = math.hypot(zr, zi if cz else 0.0)
    for k in range(lo, hi + 1):
        t = cscale2(cmul(coef(b, cc, k), pw), rho_of(k, k0, beta, rho0) - r_lo)
        acc = cadd(acc, t)
        absum += math.hypot(*(b[2 * k: 2 * k + 2] if cc else (b[k], 0.0))) * \
            2.0 ** (rho_of(k, k0, beta, rho0) - r_lo) * zabs ** (k - lo)
        pw = cmul(pw, z)
    assert S * 2.0 ** -60 <= absum * (1 + 1e-12)
    if math.isinf(E):  # values beyond the bookkeeping's range: the certificate fails
        return ok, E, S, absum
    diff = cadd(acc, (dneg(dy(out[0])), dneg(dy(out[1]))))
    # |diff| <= 2^-113 E
    Em, Ee = dy(E)
    assert abs2_le(diff, Em * Em, 2 * Ee - 226), (to_float(diff[0]), to_float(diff[1]), E)
    assert S * 2.0 ** -60 <= absum * (1 + 1e-12)
    return ok, E, S, absum


def check_rev(lib, b, cc, cz, pieces, zr, zi, lo, hi, blocks):
    k0, beta, delta, rho0, _ = pieces
    ok, out, rho, E, S = run(lib, "rev", b, cc, cz, pieces, zr, zi, lo, hi, blocks)
    assert rho == rho_of(hi, k0, beta, rho0)
    zi = zi if cz else 0.0
    z = (dy(zr), dy(zi))
    m = hi - lo
    # X = sum b_k 2^(rho(k) - rho(hi)) z^(k - lo) = exact * z^m; compare h z^m with X
    acc, pw, absum = ((0, 0), (0, 0)), ((1, 0), (0, 0)), 0.0
    r_hi = rho_of(hi, k0, beta, rho0)
    zabs = math.hypot(zr, zi)
    for k in range(lo, hi + 1):
        t = cscale2(cmul(coef(b, cc, k), pw), rho_of(k, k0, beta, rho0) - r_hi)
        acc = cadd(acc, t)
        absum += math.hypot(*(b[2 * k: 2 * k + 2] if cc else (b[k], 0.0))) * \
            2.0 ** (rho_of(k, k0, beta, rho0) - r_hi) * zabs ** (k - hi)
        pw = cmul(pw, z)
    assert S * 2.0 ** -60 <= absum * (1 + 1e-12)
    if math.isinf(E):
        return ok, E, S, absum
    # pw is z^(m + 1) after the loop: compare h z^(m + 1) with X z
    hz = cmul((dy(out[0]), dy(out[1])), pw)
    Xz = cmul(acc, z)
    diff = cadd(Xz, (dneg(hz[0]), dneg(hz[1])))
    # |h - exact| <= 2^-113 E + (m + 1) 2^-96 absum; times |z|^(m + 1)
    bound = E * 2.0 ** -113 + (m + 1) * 2.0 ** -96 * absum * (1 + 1e-9)
    bm, be = dy(bound)
    z2 = dadd(dmul(z[0], z[0]), dmul(z[1], z[1]))
    zp = (1, 0)
    for _ in range(m + 1):
        zp = dmul(zp, z2)
    B2 = dmul(dmul((bm, be), (bm, be)), zp)
    assert abs2_le(diff, B2[0], B2[1]), (E, bound)
    assert S * 2.0 ** -60 <= absum * (1 + 1e-12)
    return ok, E, S, absum


def unit_disk(n, rng, cc):
    if not cc:
        return rng.uniform(-1, 1, n)
    r = np.sqrt(rng.uniform(0, 1, n))
    ph = rng.uniform(0, 2 * math.pi, n)
    b = np.empty(2 * n)
    b[0::2] = r * np.cos(ph)
    b[1::2] = r * np.sin(ph)
    return b


# ------------------------------------------------------------ tests

def test_magnitude_helpers(lib):
    o = np.zeros(3, np.float32)
    rng = np.random.default_rng(3)
    for x in np.concatenate([2.0 ** rng.uniform(-180, 60, 400) * rng.choice([-1, 1], 400), [1.0, -0.75, 2.0 ** -186]]):
        y = float(x) * rng.uniform(-2, 2)
        lib.wc_mags(float(x), y, o.ctypes.data)
        e = math.floor(math.log2(abs(x)))
        assert o[0] == np.float32(max(2.0 ** (e + 60), 2.0 ** -126)), x  # err_mag: 2^(e(x) + 60), floor 2^-126
        ref = abs(x) * 2.0 ** 60  # mag_up: above, within 2^-19 (floor 2^-126)
        assert o[1] >= ref and o[1] <= max(ref * (1 + 2.0 ** -19), 2.0 ** -126), x
        ref = math.hypot(x, y) * 2.0 ** 60  # coef_mag_lo: below, within 2^-23 while a normal float
        assert o[2] <= ref and (ref < 2.0 ** -126 or o[2] >= ref * (1 - 2.0 ** -23)), x
    for x in (0.0, 2.0 ** -300):
        lib.wc_mags(x, 0.0, o.ctypes.data)
        assert o[0] == np.float32(2.0 ** -126) and o[1] == np.float32(2.0 ** -126) and o[2] == 0.0
    lib.wc_mags(2.0 ** 70, 0.0, o.ctypes.data)  # beyond the FP32 range: inf above, the largest float below
    assert np.isinf(o[0]) and np.isinf(o[1]) and o[2] == np.finfo(np.float32).max


@pytest.mark.parametrize("cc,cz", [(1, 1), (0, 1), (1, 0), (0, 0)])
def test_top_down_bound_holds(lib, cc, cz):
    rng = np.random.default_rng(11 + 2 * cc + cz)
    for case in range(8):
        n = int(rng.integers(20, 160))
        b = unit_disk(n, rng, cc)
        mod = 2.0 ** rng.uniform(-1.5, 0.3)
        ph = rng.uniform(0, 2 * math.pi)
        zr, zi = (mod * math.cos(ph), mod * math.sin(ph)) if cz else (mod * rng.choice([-1, 1]), 0.0)
        beta_c = -int(round(math.log2(mod)))
        pieces = make_pieces(n, rng, beta_c)
        lo = int(rng.integers(0, n // 3))
        check_top(lib, b, cc, cz, pieces, zr, zi, lo, n - 1)


@pytest.mark.parametrize("blocks", [0, 1])
@pytest.mark.parametrize("cc,cz", [(1, 1), (0, 1), (1, 0), (0, 0)])
def test_bottom_up_bound_holds(lib, cc, cz, blocks):
    rng = np.random.default_rng(31 + 4 * blocks + 2 * cc + cz)
    for case in range(6):
        n = int(rng.integers(24, 140))
        b = unit_disk(n, rng, cc)
        mod = 2.0 ** rng.uniform(-0.3, 1.5)
        ph = rng.uniform(0, 2 * math.pi)
        zr, zi = (mod * math.cos(ph), mod * math.sin(ph)) if cz else (mod * rng.choice([-1, 1]), 0.0)
        beta_c = -int(round(math.log2(mod)))
        pieces = make_pieces(n, rng, beta_c)
        hi = int(rng.integers(2 * n // 3, n))
        check_rev(lib, b, cc, cz, pieces, zr, zi, 0, hi, blocks)


def test_single_piece_long_window_blocks(lib):
    """One piece of 300 terms near |z| = 1 (the blocked bottom-up pass
    throughout, |w| <= 2.3), and |z| = 3 (single steps)."""
    rng = np.random.default_rng(5)
    n = 300
    b = unit_disk(n, rng, 1)
    pieces = (np.array([0, n], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int64),
              np.zeros((n >> LOG2_PIECE) + 2, np.int32))
    for mod in (1.05, 3.0):
        ph = rng.uniform(0, 2 * math.pi)
        ok, E, S, absum = check_rev(lib, b, 1, 1, pieces, mod * math.cos(ph), mod * math.sin(ph), 0, n - 1, 1)
        assert ok


def test_certificate_passes_random_phase_and_rejects_aligned(lib):
    """Terms of random phase away from |z| = 1: the certificate holds (E well
    below 7.6 S).  Terms of one sign at z just below 1 (a geometric series):
    the rounding errors of Horner's scheme add up over the window and the
    certificate rejects it, while its bound still holds."""
    rng = np.random.default_rng(9)
    n = 200
    pieces = (np.array([0, n], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int64),
              np.zeros((n >> LOG2_PIECE) + 2, np.int32))
    b = unit_disk(n, rng, 1)
    ok, E, S, absum = check_top(lib, b, 1, 1, pieces, 0.6, 0.3, 0, n - 1)
    assert ok and E < 4.0 * S
    # a_k = 1/3 (rounded), z = 1 - 2^-9: every partial sum positive and growing
    b = np.zeros(2 * n)
    b[0::2] = 1.0 / 3.0
    ok, E, S, absum = check_top(lib, b, 1, 1, pieces, 1.0 - 2.0 ** -9, 0.0, 0, n - 1)
    assert E > 7.6 * S  # the certificate fails: sum again exactly
    ok, E2, S2, _ = check_top(lib, b, 1, 0, pieces, 1.0 - 2.0 ** -9, 0.0, 0, n - 1)
    assert E2 > 7.6 * S2  # real z: one rounding per step, of a partial sum that grows along the window


def _step_ratios(lib, kind, cc, cz, n, rng):
    """|computed - exact| / (2^-113 bound) of single steps on random operands
    of comparable size (every rounding of the step matters)"""
    out = np.zeros(2)
    worst = 0.0
    for _ in range(n):
        hr, hm, br, bi = rng.uniform(-1, 1, 4) * 2.0 ** rng.integers(-3, 4, 4)
        if not cc:
            bi = 0.0
        if kind == "w":
            wr, wi = rng.uniform(-1.5, 1.5, 2)
            if not cz:
                wi = 0.0
            if not cc and not cz:
                hm = 0.0
            bound = lib.wc_step_w(cc, cz, hr, hm, wr, wi, br, bi, out.ctypes.data)
            w = (dy(wr), dy(wi))
        else:
            vhr, vhi = rng.uniform(-1.5, 1.5, 2)
            if not cz:
                vhi = 0.0
            vlr = vhr * rng.uniform(-1, 1) * 2.0 ** -53
            vli = vhi * rng.uniform(-1, 1) * 2.0 ** -53
            if not cc and not cz:
                hm = 0.0
            bound = lib.wc_step_v(cc, cz, hr, hm, vhr, vlr, vhi, vli, br, bi, out.ctypes.data)
            w = (dadd(dy(vhr), dy(vlr)), dadd(dy(vhi), dy(vli)))
        ex = cadd(cmul((dy(hr), dy(hm)), w), (dy(br), dy(bi)))
        diff = cadd(ex, (dneg(dy(out[0])), dneg(dy(out[1]))))
        err = math.hypot(to_float(diff[0]), to_float(diff[1]))
        assert err <= float(bound) * 2.0 ** -113 * (1 + 1e-12), (kind, cc, cz, err, bound)
        worst = max(worst, err / (float(bound) * 2.0 ** -113))
    return worst


@pytest.mark.parametrize("kind", ["w", "v"])
@pytest.mark.parametrize("cc,cz", [(1, 1), (0, 1), (1, 0), (0, 0)])
def test_single_step_bound_holds_and_is_tight(lib, kind, cc, cz):
    """Every rounding of a step is in its bound: the bound holds on random
    operands, and on some of them the error comes within a factor 2.5 of it
    (a step whose bound left out one of its roundings would be exceeded)."""
    rng = np.random.default_rng(71 + 4 * (kind == "v") + 2 * cc + cz)
    worst = _step_ratios(lib, kind, cc, cz, 3000, rng)
    assert worst > 0.4, worst


def _single_piece(n):
    return (np.array([0, n], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int64),
            np.zeros((n >> LOG2_PIECE) + 2, np.int32))


def test_blocked_pass_counts_block_sum_roundings(lib):
    """z = 1 (every multiplier exact; blocks of four), blocks whose sums
    round the same way: (1, t, t, t) rounds to 1 and (-1, t', t', t') to -1,
    t = 0.499 2^-52 and t' = 0.499 2^-53, so each block sum errs by about
    3 t or 3 t' with one sign while the partial sum G returns to 0 after
    every second block (its own roundings vanish).  The error, about
    4.5 2^-53 per pair of blocks, is then most of the bound (7 units per
    pair): a bound without the block sums' roundings (1 unit per pair)
    would fall below it."""
    B = 4
    nb = 40
    n = 1 + B * nb
    b = np.zeros(n)
    t, t2 = 0.499 * 2.0 ** -52, 0.499 * 2.0 ** -53
    for m in range(nb):
        k0 = 1 + B * m  # block sum over b[k0 .. k0 + B - 1], the top index first
        if m % 2 == 0:
            b[k0 + B - 1], b[k0:k0 + B - 1] = 1.0, t
        else:
            b[k0 + B - 1], b[k0:k0 + B - 1] = -1.0, t2
    ok, E, S, absum = check_rev(lib, b, 0, 0, _single_piece(n), 1.0, 0.0, 0, n - 1, 1)
    _, out, _, E2, _ = run(lib, "rev", b, 0, 0, _single_piece(n), 1.0, 0.0, 0, n - 1, 1)
    err = abs(math.fsum([*b]) - out[0])  # z = 1: the window sum is the plain sum (fsum: exact here)
    assert err > 0.5 * E2 * 2.0 ** -113, (err, E2)
