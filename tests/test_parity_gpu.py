"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Windows must equal the oracle's up to boundary ties; values must satisfy
|P_gpu - P_ref| <= 2^-50 S(z) with S(z) = sum |a_k||z|^k (p = 53), checked on
every point against the oracle's window sum (with the window's own S, a
stricter scale) and on sampled points against the oracle's full Horner sum.
"""
import math
import zlib

import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TOL_FP32, TOL_FP64, error_ratio, windows_agree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_06320_gb300 as F
    F._load()
    return torch, F


def run_gpu(env, coef, zre, zim, p=53, flags=0):
    torch, F = env
    P = F.fpe_precondition(coef.re, coef.im, coef.e2, p, flags)
    n = zre.shape[0]
    zr = torch.from_numpy(np.ascontiguousarray(zre)).cuda()
    zi = None if zim is None else torch.from_numpy(np.ascontiguousarray(zim)).cuda()
    out = F.empty_out(n)
    nt = torch.empty(n, dtype=torch.int32, device="cuda")
    bl = torch.empty(n, dtype=torch.int32, device="cuda")
    F.fpe_eval(P, zr, zi, out, nt, bl)
    l, r, N = F.fpe_get_windows(P, n)
    F.fpe_sync(P)
    return P, out.cpu().numpy(), nt.cpu().numpy(), l.cpu().numpy(), r.cpu().numpy(), N.cpu().numpy()


def sample_indices(n, lengths, lam, k=256, seed=0):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(n, size=min(n, k), replace=False).tolist())
    fin = np.nonzero(np.isfinite(lam))[0]
    idx |= set(fin[np.argsort(-lengths[fin])[:64]].tolist())          # longest windows
    idx |= set(fin[np.argsort(np.abs(lam[fin]))[:64]].tolist())       # closest to |z| = 1
    return np.array(sorted(idx))


def check_workload(env, coef, pts, p=53, n_full=256, tol=TOL_FP64, check_full=True, flags=0):
    P, out, nt, l, r, N = run_gpu(env, coef, pts.re, pts.im, p, flags)
    pre = oracle.precondition(coef, p)
    lam = oracle.log2_abs(pts.re, pts.im)
    kl, No, Lo, Ro = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    fin = np.isfinite(lam)
    # windows (def. LRN)
    agree = windows_agree(l[fin], r[fin], Lo[fin], Ro[fin], pre.hk, pre.hs, pre.T, lam[fin], No[fin])
    assert agree.all(), f"{(~agree).sum()} windows differ beyond boundary ties"
    assert np.allclose(N[fin], No[fin], rtol=1e-12, atol=1e-9)
    # kept-term counts
    same = fin.copy()
    same[fin] = (l[fin] == Lo[fin]) & (r[fin] == Ro[fin])
    cg = np.concatenate([[0], np.cumsum(pre.good)])
    want_nt = cg[np.minimum(Ro, pre.d) + 1] - cg[Lo]
    assert np.array_equal(nt[same], want_nt[same])
    # values against the window sum over the oracle's windows, every point
    L2, R2 = Lo.copy(), Ro.copy()
    L2[~fin], R2[~fin] = 0, 0
    Q, SQ = oracle.window_sum(coef, pre.good, pts.re, pts.im, L2, R2, with_S=True)
    ratio = error_ratio(out, Q, SQ, tol * 31 / 32)
    worst = int(np.argmax(ratio))
    assert ratio.max() <= 1.0, f"point {worst}: error {ratio.max():.3g} x tolerance (window sum)"
    stats = {"max_ratio_window": float(ratio.max()), "median_ratio_window": float(np.median(ratio))}
    if check_full:
        idx = sample_indices(pts.n, Ro - Lo + 1, lam, k=n_full)
        ref, S, _ = oracle.horner_ref(coef, pts.re[idx], None if pts.im is None else pts.im[idx])
        rf = error_ratio(out[idx], ref, S, tol)
        assert rf.max() <= 1.0, f"point {idx[int(np.argmax(rf))]}: error {rf.max():.3g} x tolerance (full Horner)"
        stats["max_ratio_full"] = float(rf.max())
    return stats


# --------------------------------------------------------------- workloads

def test_unit_square_d1000_all_points(env):
    """d=1000, a_k = x+iy with x, y ~ U[-1,1] (seed 0), 10^4 sphere points:
    every point against the full Horner reference."""
    wl = W.unit_square_d1000()
    st = check_workload(env, wl.coeffs, wl.points, n_full=wl.points.n)
    print("unit_square_d1000", st)


def test_unit_disk_d2pow20_full_size(env):
    """The headline workload at full size: d=2^20, 2^20 sphere points."""
    wl = W.unit_disk_d2pow20()
    st = check_workload(env, wl.coeffs, wl.points, n_full=384)
    print("unit_disk_d2pow20", st)


def test_inverse_factorial(env):
    wl = W.inverse_factorial_d1e5(n_points=1 << 15)
    st = check_workload(env, wl.coeffs, wl.points, n_full=128)
    print("inverse_factorial", st)


def test_mandelbrot(env):
    wl = W.mandelbrot_real(11, n_points=1 << 15)
    st = check_workload(env, wl.coeffs, wl.points, n_full=256)
    print("mandelbrot_n11", st)


def test_mandelbrot_n20(env):
    """The Mandelbrot iterate at n = 20 (d = 2^20, coefficients up to 2^616226),
    2^14 real points in [-2, 0.25]."""
    wl = W.mandelbrot_real(20, n_points=1 << 14)
    st = check_workload(env, wl.coeffs, wl.points, n_full=16)
    print("mandelbrot_n20", st)


def test_sparse_d2pow22(env):
    wl = W.sparse_d2pow22(n_points=1 << 15)
    st = check_workload(env, wl.coeffs, wl.points, n_full=24)
    print("sparse", st)


FAMILIES = ["half_circle", "half_circle_complex", "chebyshev", "geometric", "lognormal", "ext_random",
            "real_coef_complex_pts", "complex_coef_real_pts", "trimmed", "sparse_small"]


# Both modes meet the tolerance on every family: the default mode's FP64 window
# sums carry rounding-error certificates, and a window whose certificate fails
# (aligned terms of the geometric series near z = 1, for one) is summed again
# exactly on the integer pipe.
@pytest.mark.parametrize("accurate", [False, True], ids=["default", "accurate"])
@pytest.mark.parametrize("family", FAMILIES)
def test_families(env, family, accurate):
    torch, F = env
    rng = np.random.default_rng(zlib.crc32(family.encode()))
    n = 4096
    if family == "half_circle":
        coef, pts = W.half_circle(1000), W.sphere_points(n, rng)
    elif family == "half_circle_complex":
        coef, pts = W.half_circle(1000, True, rng), W.sphere_points(n, rng)
    elif family == "chebyshev":
        coef, pts = W.chebyshev_T(300), W.real_line_points(n, -1.2, 1.2, rng)
    elif family == "geometric":
        coef, pts = W.geometric(3000), W.disk_points(n, rng)
    elif family == "lognormal":
        coef, pts = W.lognormal_profile(20000, 0.005, rng), W.sphere_points(n, rng)
    elif family == "ext_random":
        e2 = rng.integers(-3000, 3000, 500)
        coef, pts = W.Coeffs(rng.uniform(-1, 1, 500), rng.uniform(-1, 1, 500), e2), W.sphere_points(n, rng)
    elif family == "real_coef_complex_pts":
        coef, pts = W.Coeffs(rng.uniform(-1, 1, 5000)), W.sphere_points(n, rng)
    elif family == "complex_coef_real_pts":
        coef, pts = W.unit_disk_complex(5000, rng), W.real_circle_points(n, rng)
    elif family == "sparse_small":
        coef, pts = W.sparse_real(20000, 0.02, rng), W.sphere_points(n, rng)
    else:
        coef = W.unit_square_complex(2000, rng)
        coef.re[:13] = 0
        coef.im[:13] = 0
        coef.re[-9:] = 0
        coef.im[-9:] = 0
        pts = W.sphere_points(n, rng)
    st = check_workload(env, coef, pts, n_full=128, flags=F.FPE_ACCURATE if accurate else 0)
    print(family, "accurate" if accurate else "default", st)


@pytest.mark.parametrize("name", ["unit_square_d1000", "inverse_factorial", "mandelbrot", "sparse"])
def test_workloads_accurate_mode(env, name):
    torch, F = env
    if name == "unit_square_d1000":
        wl = W.unit_square_d1000()
    elif name == "inverse_factorial":
        wl = W.inverse_factorial_d1e5(n_points=1 << 14)
    elif name == "mandelbrot":
        wl = W.mandelbrot_real(11, n_points=1 << 14)
    else:
        wl = W.sparse_d2pow22(n_points=1 << 14)
    st = check_workload(env, wl.coeffs, wl.points, n_full=64, flags=F.FPE_ACCURATE)
    print(name, "accurate", st)


def test_worked_example_windows(env):
    """§4.1 example: moduli exactly 2^(s_k - 1) (phases on the axes), the
    algorithm's T = p + s(d) + 3 = 13 at p = 6, points at exactly |z| = 1 and
    |z| = 2^-3.  Hand-derived windows for T = 13: [4, 10] at lambda = 0 and
    [0, 9] at lambda = -3."""
    rng = np.random.default_rng(5)
    s = np.array(W.worked_example_scales())
    ph = rng.integers(0, 4, s.size)
    re = np.choose(ph, [1.0, 0.0, -1.0, 0.0])
    im = np.choose(ph, [0.0, 1.0, 0.0, -1.0])
    coef = W.Coeffs(re, im, s - 1)
    zre = np.array([1.0, 0.0, -1.0, 0.0, 0.125, 0.0, -0.125, 0.0])
    zim = np.array([0.0, 1.0, 0.0, -1.0, 0.0, 0.125, 0.0, -0.125])
    P, out, nt, l, r, N = run_gpu(env, coef, zre, zim, p=6)
    pre = oracle.precondition(coef, 6)
    assert pre.T == 13
    assert list(pre.hk) == [0, 1, 3, 6, 8, 9, 10]
    lam = oracle.log2_abs(zre, zim)
    _, No, Lo, Ro = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    assert list(l) == list(Lo) == [4, 4, 4, 4, 0, 0, 0, 0]
    assert list(r) == list(Ro) == [10, 10, 10, 10, 9, 9, 9, 9]
    assert list(N) == [30.0] * 4 + [9.0] * 4
    # random phases: |e^{i phi}| rounds to 1 +- ulp, so boundary ties may go either way
    ph = rng.uniform(0, 2 * math.pi, 64)
    mod = np.where(np.arange(64) % 2 == 0, 1.0, 0.125)
    pts = W.Points(mod * np.cos(ph), mod * np.sin(ph))
    check_workload(env, coef, pts, p=6, n_full=0, check_full=False, tol=2.0 ** -50)


# --------------------------------------------------------------- edge cases

def test_edge_points(env):
    torch, F = env
    rng = np.random.default_rng(77)
    coef = W.unit_square_complex(700, rng)
    zre = np.array([0.0, 1e-300, 1e300, 5e-324, 1.0, -1.0, 0.0, 2.0 ** 40, 2.0 ** -40, 1.0 + 2 ** -52])
    zim = np.array([0.0, 0.0, -1e300, 0.0, 0.0, 0.0, 1.0, 2.0 ** 40, 0.0, 0.0])
    st = check_workload(env, coef, W.Points(zre, zim), n_full=zre.size)
    # z = 0 returns a_0
    P, out, *_ = run_gpu(env, coef, zre[:1], zim[:1])
    e = np.ascontiguousarray(out[:, 2]).view(np.int64)[0]
    assert out[0, 0] * 2.0 ** float(e) == coef.re[0] and out[0, 1] * 2.0 ** float(e) == coef.im[0]


def test_zero_point_with_positive_valuation(env):
    coef = W.Coeffs(np.array([0.0, 0.0, 1.5, -2.0]), np.array([0.0, 0.0, 0.5, 1.0]))
    P, out, nt, *_ = run_gpu(env, coef, np.array([0.0, 0.5]), np.array([0.0, 0.25]))
    assert out[0, 0] == 0.0 and out[0, 1] == 0.0 and nt[0] == 0
    ref, S, _ = oracle.horner_ref(coef, np.array([0.5]), np.array([0.25]))
    assert error_ratio(out[1:], ref, S).max() <= 1.0


def test_constant_and_linear(env):
    for coef in (W.Coeffs(np.array([-3.25])), W.Coeffs(np.array([1.0, 1.0])),
                 W.Coeffs(np.array([2.0]), np.array([-7.0]))):
        rng = np.random.default_rng(3)
        pts = W.sphere_points(2000, rng)
        check_workload(env, coef, pts, n_full=2000)


def test_nonfinite_points_flagged(env):
    torch, F = env
    coef = W.unit_square_complex(100, np.random.default_rng(1))
    P = F.fpe_precondition(coef.re, coef.im)
    z = torch.tensor([0.5, float("nan"), float("inf"), 0.25], dtype=torch.float64, device="cuda")
    zi = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = F.fpe_eval(P, z, zi)
    with pytest.raises(F.FpeError) as e:
        F.fpe_sync(P)
    assert e.value.status == F.FPE_ERR_NONFINITE
    o = out.cpu().numpy()
    assert np.isnan(o[1, 0]) and np.isnan(o[2, 0]) and np.isfinite(o[0, 0]) and np.isfinite(o[3, 0])
    F.fpe_sync(P)  # status cleared


def test_empty_and_single_point(env):
    torch, F = env
    coef = W.unit_square_complex(100, np.random.default_rng(2))
    P = F.fpe_precondition(coef.re, coef.im)
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = F.fpe_eval(P, z, z)
    F.fpe_sync(P)
    assert out.shape == (0, 3)
    check_workload(env, coef, W.Points(np.array([0.9]), np.array([0.3])), n_full=1)


def test_host_buffers_match_device(env):
    torch, F = env
    wl = W.unit_square_d1000(n_points=5000)
    P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im)
    out_h, nt_h, bl_h = F.fpe_eval_host(P, wl.points.re, wl.points.im, want_diag=True)
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = torch.from_numpy(wl.points.im).cuda()
    out_d = F.fpe_eval(P, zr, zi).cpu().numpy()
    # compare bit patterns (the exponent column holds int64 bits)
    assert np.array_equal(out_h.view(np.int64), out_d.view(np.int64))


# --------------------------------------------------------------- Horner baselines

@pytest.mark.parametrize("compensated", [False, True])
def test_horner_baselines(env, compensated):
    torch, F = env
    wl = W.unit_square_d1000(n_points=2000)
    P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im)
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = torch.from_numpy(wl.points.im).cuda()
    out = F.fpe_horner(P, zr, zi, compensated=compensated).cpu().numpy()
    F.fpe_sync(P)
    ref, S, _ = oracle.horner_ref(wl.coeffs, wl.points.re, wl.points.im)
    r = error_ratio(out, ref, S)
    print("horner", "compensated" if compensated else "plain", "max ratio", r.max(), "median", np.median(r))
    if compensated:
        assert r.max() <= 1.0
    else:
        assert np.median(r) <= 1.0 and np.all(np.isfinite(r))


def test_horner_compensated_large_degree(env):
    torch, F = env
    wl = W.unit_disk_d2pow20(n_points=64)
    P = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im)
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = torch.from_numpy(wl.points.im).cuda()
    out = F.fpe_horner(P, zr, zi, compensated=True).cpu().numpy()
    F.fpe_sync(P)
    ref, S, _ = oracle.horner_ref(wl.coeffs, wl.points.re, wl.points.im)
    assert error_ratio(out, ref, S).max() <= 1.0


# --------------------------------------------------------------- derivative, batch

def test_derivative(env):
    """P'(z) from the separately preconditioned k a_k (§7.2) against the oracle's
    Horner on the exact derivative coefficients (k a_k exactly, as double-double)."""
    torch, F = env
    rng = np.random.default_rng(8)
    coef = W.unit_square_complex(1500, rng)
    pts = W.sphere_points(3000, rng)
    P = F.fpe_precondition(coef.re, coef.im, None, 53, F.FPE_WITH_DERIV)
    zr = torch.from_numpy(pts.re).cuda()
    zi = torch.from_numpy(pts.im).cuda()
    out = F.fpe_eval_deriv(P, zr, zi).cpu().numpy()
    F.fpe_sync(P)
    k = np.arange(1, coef.n_coef, dtype=np.float64)
    # exact k a_k as (hi, lo): k < 2^11 and |a| < 1, split via two products
    hi_r = k * coef.re[1:]
    hi_i = k * coef.im[1:]
    from fractions import Fraction
    lo_r = np.array([float(Fraction(float(a)) * int(b) - Fraction(float(h))) for a, b, h in zip(coef.re[1:], k, hi_r)])
    lo_i = np.array([float(Fraction(float(a)) * int(b) - Fraction(float(h))) for a, b, h in zip(coef.im[1:], k, hi_i)])
    dcoef = W.Coeffs(hi_r, hi_i)
    ref, S, _ = oracle.horner_ref(dcoef, pts.re, pts.im, coef_lo=(lo_r, lo_i))
    assert error_ratio(out, ref, S).max() <= 1.0


def test_batch_matches_single(env):
    torch, F = env
    rng = np.random.default_rng(10)
    wls = W.batched_lognormal(n_poly=12, pts_per_poly=300, seed=3, dmin=16, dmax=5000)
    polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im) for w in wls]
    offs = np.concatenate([[0], np.cumsum([w.points.n for w in wls])])
    zre = np.concatenate([w.points.re for w in wls])
    zim = np.concatenate([w.points.im for w in wls])
    out = F.fpe_eval_batch(polys, offs, torch.from_numpy(zre).cuda(), torch.from_numpy(zim).cuda()).cpu().numpy()
    for i, w in enumerate(wls):
        ref, S, _ = oracle.horner_ref(w.coeffs, w.points.re, w.points.im)
        assert error_ratio(out[offs[i]:offs[i + 1]], ref, S).max() <= 1.0


def test_long_windows_group_overflow(env):
    """Every point on the unit circle: every window is the whole polynomial
    (4 warp groups each), more extra group slots than the scratch holds, so
    most points fall back to one group per window; results stay exact."""
    rng = np.random.default_rng(12)
    coef = W.unit_disk_complex((1 << 17) - 1, rng)
    t = rng.uniform(0, 2 * math.pi, 2048)
    pts = W.Points(np.cos(t), np.sin(t))
    st = check_workload(env, coef, pts, n_full=0, check_full=False)
    print("unit circle, d=2^17-1", st)


# --------------------------------------------------------------- FP32 mode (p = 24)

@pytest.mark.parametrize("name", ["unit_square_d1000", "unit_disk_d2pow20", "inverse_factorial", "mandelbrot",
                                  "half_circle_complex", "lognormal", "real_coef_complex_pts",
                                  "complex_coef_real_pts", "unit_circle"])
def test_fp32_mode(env, name):
    """FPE_FP32: windows and G_p at p = 24, FP32 coefficients and Horner on the
    FP32 pipe; |P_gpu - P_ref| <= 2^-21 S(z)."""
    torch, F = env
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    n_full = 128
    if name == "unit_square_d1000":
        wl = W.unit_square_d1000()
        coef, pts = wl.coeffs, wl.points
    elif name == "unit_disk_d2pow20":
        wl = W.unit_disk_d2pow20(n_points=1 << 18)
        coef, pts = wl.coeffs, wl.points
        n_full = 96
    elif name == "inverse_factorial":
        wl = W.inverse_factorial_d1e5(n_points=1 << 14)
        coef, pts = wl.coeffs, wl.points
    elif name == "mandelbrot":
        wl = W.mandelbrot_real(11, n_points=1 << 14)
        coef, pts = wl.coeffs, wl.points
    elif name == "half_circle_complex":
        coef, pts = W.half_circle(1000, True, rng), W.sphere_points(4096, rng)
    elif name == "lognormal":
        coef, pts = W.lognormal_profile(20000, 0.005, rng), W.sphere_points(4096, rng)
    elif name == "real_coef_complex_pts":
        coef, pts = W.Coeffs(rng.uniform(-1, 1, 5000)), W.sphere_points(4096, rng)
    elif name == "complex_coef_real_pts":
        coef, pts = W.unit_disk_complex(5000, rng), W.real_circle_points(4096, rng)
    else:
        coef = W.unit_disk_complex((1 << 16) - 1, rng)
        t = rng.uniform(0, 2 * math.pi, 1024)
        pts = W.Points(np.cos(t), np.sin(t))
        n_full = 16
    st = check_workload(env, coef, pts, p=24, n_full=n_full, tol=TOL_FP32, flags=F.FPE_FP32)
    print("fp32", name, st)


def test_fp32_flags(env):
    torch, F = env
    c = W.unit_square_complex(10, np.random.default_rng(0))
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(c.re, c.im, None, 53, F.FPE_FP32)
    assert e.value.status == F.FPE_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["unit_square_d1000", "inverse_factorial"])
def test_bits_lost_diagnostic(env, name):
    """bits_lost = max(0, ceil(N) - e) estimates the leading bits cancelled in
    the computed value (the confidence estimator of §4.1; the remark on
    cancellations in §2.5).  Where the cancellation c = log2(max_k |a_k z^k|)
    - log2|P(z)| is moderate the output carries |P| to a few bits, so
    bits_lost is within 2 of c (N within 1 of the largest term's log2, e
    within 1 of log2|P|).  Past about 50 bits the FP64 output sits at the
    error floor 2^-50 sum |a_k z^k|, so bits_lost saturates near 50 minus
    log2 of the window length, and only its lower bound is checked."""
    torch, F = env
    if name == "unit_square_d1000":
        wl = W.unit_square_d1000(n_points=2000)
    else:
        wl = W.inverse_factorial_d1e5(n_points=2000, d=3000)
    P, out, nt, l, r, N = run_gpu(env, wl.coeffs, wl.points.re, wl.points.im)
    zr = torch.from_numpy(wl.points.re).cuda()
    zi = None if wl.points.im is None else torch.from_numpy(wl.points.im).cuda()
    bl = torch.empty(wl.points.n, dtype=torch.int32, device="cuda")
    F.fpe_eval(P, zr, zi, bits_lost=bl)
    F.fpe_sync(P)
    bl = bl.cpu().numpy()
    ref, S, l2M = oracle.horner_ref(wl.coeffs, wl.points.re, wl.points.im)
    mag = np.hypot(ref.re_hi + ref.re_lo, ref.im_hi + ref.im_lo)
    l2P = np.log2(mag) + ref.e
    want = np.maximum(0.0, l2M - l2P)
    floor_bits = 50 - np.log2(np.maximum(nt, 1))
    moderate = want <= floor_bits - 6
    assert np.all(np.abs(bl[moderate] - want[moderate]) <= 2.0)
    assert np.all(bl[~moderate] >= floor_bits[~moderate] - 8)
    if name == "inverse_factorial":
        assert bl.max() > 30  # e^x at x ~ -50 cancels ~144 bits in the sum


@pytest.mark.parametrize("case", ["dense_forced_sparse", "sparse_forced_dense"])
def test_forced_window_sum_kind(env, case):
    """FPE_FORCE_SPARSE sums every window over its good indices alone (on a
    dense polynomial: all windows); FPE_FORCE_DENSE never does (on a sparse
    one: Horner over every index, zeros included, with the certificates).
    Both meet the tolerance."""
    torch, F = env
    if case == "dense_forced_sparse":
        wl = W.unit_square_d1000(n_points=4096)
        flags = F.FPE_FORCE_SPARSE
    else:
        wl = W.sparse_d2pow22(n_points=1 << 13)
        flags = F.FPE_FORCE_DENSE
    st = check_workload(env, wl.coeffs, wl.points, n_full=48, flags=flags)
    print(case, st)

