"""Tensor-core window sums (fpe_set_tensor_path): parity against the oracle on
the workloads that take the path, bit-for-bit reproducibility, the hand-back
of wide groups to the FP64 kernels, work items split across several CTAs,
a piece with a nonzero integer slope, real coefficients and real points.

Every window the path sums is compared with the oracle's window sum (its own
S, the stricter scale) and sampled points with the full Horner reference, at
|P_gpu - P_ref| <= 2^-50 S(z)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TOL_FP64, error_ratio

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_06320_gb300 as F
    F._load()
    return torch, F


def _eval(env, P, zre, zim):
    torch, F = env
    n = zre.shape[0]
    zr = torch.from_numpy(np.ascontiguousarray(zre)).cuda()
    zi = None if zim is None else torch.from_numpy(np.ascontiguousarray(zim)).cuda()
    out = F.empty_out(n)
    nt = torch.empty(n, dtype=torch.int32, device="cuda")
    F.fpe_eval(P, zr, zi, out, nt)
    F.fpe_sync(P)
    return out.cpu().numpy(), nt.cpu().numpy(), F.fpe_tensor_stats(P)


def _check(env, coef, zre, zim, n_full=128, min_tc_points=1, min_window=64):
    """Tensor path on for windows of at least min_window terms (64: more
    points than the default takes, down to one block per window): values vs
    the oracle (window sums on every point, full Horner on a sample); returns
    the stats and the outputs."""
    torch, F = env
    P = F.fpe_precondition(coef.re, coef.im, coef.e2, 53)
    assert F.fpe_get_tensor_path(P)["pieces"] >= 1
    F.fpe_set_tensor_path(P, min_window)
    out, nt, st = _eval(env, P, zre, zim)
    assert st["points"] >= min_tc_points, st
    pre = oracle.precondition(coef, 53)
    lam = oracle.log2_abs(zre, zim)
    _, _, Lo, Ro = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    Q, SQ = oracle.window_sum(coef, pre.good, zre, zim, Lo, Ro, with_S=True)
    r = error_ratio(out, Q, SQ, TOL_FP64 * 31 / 32)
    assert r.max() <= 1.0, f"window sums: {r.max():.3g} x tolerance at point {int(np.argmax(r))}"
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.choice(zre.shape[0], min(n_full, zre.shape[0]), replace=False),
                                    np.argsort(-(Ro - Lo))[:16]]))
    ref, S, _ = oracle.horner_ref(coef, zre[idx], None if zim is None else zim[idx])
    rf = error_ratio(out[idx], ref, S, TOL_FP64)
    assert rf.max() <= 1.0, f"full Horner: {rf.max():.3g} x tolerance"
    cg = np.concatenate([[0], np.cumsum(pre.good)])
    assert np.array_equal(nt, cg[np.minimum(Ro, pre.d) + 1] - cg[Lo])
    return P, st, out


def _flat_disk(d, rng):
    """Coefficients uniform in the unit disk with |a_0| = |a_d| = 0.9, so that
    s(a_0) = s(a_d) = 0 is the largest scale and the cover is one flat piece
    (the path only takes windows inside one piece with an integer slope)."""
    c = W.unit_disk_complex(d, rng)
    for k in (0, d):
        r = math.hypot(c.re[k], c.im[k]) or 1.0
        c.re[k], c.im[k] = 0.9 * c.re[k] / r, 0.9 * c.im[k] / r
    return c


def test_sphere_points_unit_disk(env):
    rng = np.random.default_rng(101)
    coef = _flat_disk(1 << 16, rng)
    pts = W.sphere_points(1 << 15, rng)
    _, st, _ = _check(env, coef, pts.re, pts.im, min_tc_points=1 << 13)
    assert st["tiles"] >= 1 and st["subtiles"] >= st["items"] >= st["tiles"]


def test_default_threshold(env):
    """The default setting (windows of 384 terms or more) on sphere points;
    a call below 32768 points leaves the path off unless it was set."""
    torch, F = env
    rng = np.random.default_rng(108)
    coef = _flat_disk(1 << 16, rng)
    pts = W.sphere_points(1 << 14, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    assert F.fpe_get_tensor_path(P)["min_window"] == 384
    _, _, st = _eval(env, P, pts.re, pts.im)
    assert st["points"] == 0  # 2^14 points: below the default's size rule
    big = W.sphere_points(1 << 15, rng)
    _, _, st = _eval(env, P, big.re, big.im)
    assert st["points"] > 0
    _check(env, coef, pts.re, pts.im, min_tc_points=512, min_window=384)


def test_reproducible_and_same_as_fp64_path(env):
    """Two calls give the same bits; the FP64 kernels (path off) agree within
    the tolerance and count the same kept terms."""
    torch, F = env
    rng = np.random.default_rng(102)
    coef = _flat_disk(3000, rng)
    pts = W.sphere_points(20000, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    F.fpe_set_tensor_path(P, 384)  # the default threshold, on a call below the default's 32768 points
    a, nta, st = _eval(env, P, pts.re, pts.im)
    b, _, _ = _eval(env, P, pts.re, pts.im)
    assert st["points"] > 0
    assert np.array_equal(a.view(np.int64), b.view(np.int64))
    F.fpe_set_tensor_path(P, 0)
    c, ntc, st0 = _eval(env, P, pts.re, pts.im)
    assert st0["points"] == 0
    assert np.array_equal(nta, ntc)
    _, S, _ = oracle.horner_ref(coef, pts.re, pts.im)
    ce = np.ascontiguousarray(c[:, 2]).view(np.int64)
    ref = oracle.ExtValues(np.stack([c[:, 0], np.zeros(len(c)), c[:, 1], np.zeros(len(c))], axis=1), ce)
    assert error_ratio(a, ref, S, TOL_FP64).max() <= 1.0


def test_long_windows_several_items(env):
    """|z| within 2^-12 of 1 at d = 2^18: windows of ~2^18 terms, cut into
    several work items per tile and joined by the finalize kernel."""
    torch, F = env
    rng = np.random.default_rng(103)
    coef = _flat_disk(1 << 18, rng)
    n = 2048
    lam = rng.uniform(-2.0 ** -12, 2.0 ** -12, n)
    th = rng.uniform(0, 2 * math.pi, n)
    zre, zim = 2.0 ** lam * np.cos(th), 2.0 ** lam * np.sin(th)
    _, st, _ = _check(env, coef, zre, zim, n_full=24, min_tc_points=n)
    assert st["items"] > st["tiles"], st


def test_sparse_points_handed_back(env):
    """A few points spread over |z| in [1/4, 4]: groups too wide for one tilt
    go back to the FP64 kernels, and every value is still right."""
    rng = np.random.default_rng(104)
    coef = _flat_disk(5000, rng)
    n = 300
    lam = rng.uniform(-2.0, 2.0, n)
    th = rng.uniform(0, 2 * math.pi, n)
    zre, zim = 2.0 ** lam * np.cos(th), 2.0 ** lam * np.sin(th)
    torch, F = env
    P, st, _ = _check(env, coef, zre, zim, n_full=64, min_tc_points=0)
    assert st["rejected"] > 0, st


def test_nonzero_integer_slope_piece(env):
    """Scales flat (a_k ~ 1) up to k = 3000, then falling one bit per index:
    for |z| > 2 the windows lie in the second piece (beta = -1)."""
    rng = np.random.default_rng(105)
    d = 8000
    k = np.arange(d + 1)
    mod = np.sqrt(rng.uniform(0.25, 1.0, d + 1))  # s(a_k) = 0 before the exponent
    ph = rng.uniform(0, 2 * math.pi, d + 1)
    e2 = np.where(k <= 3000, 0, -(k - 3000)).astype(np.int64)  # a_k = mantissa 2^e2: no underflow
    coef = W.Coeffs(mod * np.cos(ph), mod * np.sin(ph), e2)
    n = 8192
    lam = np.concatenate([rng.uniform(-0.05, -0.001, n // 2), rng.uniform(1.001, 1.05, n // 2)])
    th = rng.uniform(0, 2 * math.pi, n)
    zre, zim = 2.0 ** lam * np.cos(th), 2.0 ** lam * np.sin(th)
    torch, F = env
    P, st, _ = _check(env, coef, zre, zim, n_full=64, min_tc_points=n // 4)
    assert F.fpe_get_tensor_path(P)["pieces"] >= 2


def test_real_coefficients_complex_and_real_points(env):
    """Real coefficients (one column of the slices is zero), at complex and at
    real points (the imaginary slices of the powers are zero)."""
    rng = np.random.default_rng(106)
    d = 20000
    a = rng.uniform(-1, 1, d + 1)
    a[0], a[d] = 0.9, -0.9  # the largest scale at both ends: one flat piece
    coef = W.Coeffs(a)
    pts = W.sphere_points(8192, rng)
    _check(env, coef, pts.re, pts.im, n_full=64, min_tc_points=1000)
    x = np.concatenate([rng.uniform(-1.02, -0.98, 2048), rng.uniform(0.98, 1.02, 2048)])
    _check(env, coef, x, None, n_full=64, min_tc_points=1000)


def test_geometric_series_default_mode(env):
    """All a_k = 1 near z = 1 (aligned terms): the FP64 window kernels need
    FPE_ACCURATE here, the exact slice products do not."""
    rng = np.random.default_rng(107)
    d = 1 << 14
    coef = W.geometric(d)
    n = 2048
    lam = rng.uniform(-2.0 ** -6, 2.0 ** -6, n)
    th = rng.uniform(-0.01, 0.01, n)
    zre, zim = 2.0 ** lam * np.cos(th), 2.0 ** lam * np.sin(th)
    _check(env, coef, zre, zim, n_full=64, min_tc_points=n // 2)
