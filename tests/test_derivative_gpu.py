"""Derivatives on the FPE path (§7.2): P', the Newton step, and the gradients
behind the torch.autograd.Function, against the oracle, the paper's FP32
Newton example, a dense gradient and finite differences."""
import math
from fractions import Fraction

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


def _xc64_complex(out):
    e = np.ascontiguousarray(out[:, 2]).view(np.int64)
    return out[:, 0], out[:, 1], e


def _deriv_coef_exact(coef):
    """k a_k exactly, as (hi, lo) double pairs (k < 2^20, so the product fits 106 bits)."""
    k = np.arange(1, coef.n_coef)
    hr = k * coef.re[1:]
    hi_ = k * coef.im[1:] if coef.im is not None else None
    lr = np.array([float(Fraction(float(a)) * int(b) - Fraction(float(h))) for a, b, h in zip(coef.re[1:], k, hr)])
    li = (np.array([float(Fraction(float(a)) * int(b) - Fraction(float(h)))
                    for a, b, h in zip(coef.im[1:], k, hi_)]) if hi_ is not None else None)
    return W.Coeffs(hr, hi_), (lr, li)


@pytest.mark.parametrize("fp32", [True, False], ids=["fp32_p24", "fp64_p53"])
def test_newton_paper_example(env, fp32):
    """P(z) = z^64 + 1 at z = 10 (end of §7.2): P(10) and P'(10) overflow FP32,
    yet the increment 10 - N_P(10) = 0.15625 + 1.5625e-65 comes out right."""
    torch, F = env
    c = np.zeros(65)
    c[0] = c[64] = 1.0
    flags = F.FPE_WITH_DERIV | (F.FPE_FP32 if fp32 else 0)
    P = F.fpe_precondition(c, None, None, 24 if fp32 else 53, flags)
    z = torch.tensor([10.0], dtype=torch.float64, device="cuda")
    inc, zn, _ = F.fpe_newton(P, z)
    F.fpe_sync(P)
    re, im, e = _xc64_complex(inc.cpu().numpy())
    val = re[0] * 2.0 ** int(e[0])
    tol = 2.0 ** -21 if fp32 else 2.0 ** -50
    assert abs(val - 0.15625) <= tol * 0.15625 and im[0] == 0.0
    assert abs(zn.item() - (10.0 - 0.15625)) <= tol * 10
    # and P(10) itself is represented, far beyond the FP32 range
    v = F.fpe_eval(P, z).cpu().numpy()
    re, im, e = _xc64_complex(v)
    assert abs(math.log2(abs(re[0])) + int(e[0]) - 64 * math.log2(10)) < 1e-6


def test_newton_and_point_gradient_vs_oracle(env):
    torch, F = env
    rng = np.random.default_rng(21)
    coef = W.unit_square_complex(500, rng)
    pts = W.sphere_points(2000, rng)
    P = F.fpe_precondition(coef.re, coef.im, None, 53, F.FPE_WITH_DERIV)
    zr = torch.from_numpy(pts.re).cuda()
    zi = torch.from_numpy(pts.im).cuda()
    inc, znr, zni = F.fpe_newton(P, zr, zi)
    g = rng.normal(size=(2, pts.n))
    gz_re, gz_im = F.fpe_grad_points(P, zr, zi, torch.from_numpy(g[0]).cuda(), torch.from_numpy(g[1]).cuda())
    F.fpe_sync(P)
    ref, S, _ = oracle.horner_ref(coef, pts.re, pts.im)
    dcoef, dlo = _deriv_coef_exact(coef)
    dref, dS, _ = oracle.horner_ref(dcoef, pts.re, pts.im, coef_lo=dlo)
    # everything as mantissa x 2^exponent: P = Pm 2^eP, P' = Dm 2^eD
    Pm = (ref.re_hi + ref.re_lo) + 1j * (ref.im_hi + ref.im_lo)
    Dm = (dref.re_hi + dref.re_lo) + 1j * (dref.im_hi + dref.im_lo)
    eP, eD = ref.e, dref.e
    ok = (np.abs(Dm) > 0) & (np.abs(Pm) > 0)
    qm = np.where(ok, Pm / np.where(ok, Dm, 1.0), 0.0)
    qe = eP - eD
    ldx = lambda m, e: np.ldexp(m, np.clip(e, -1000, 1000).astype(np.int32))
    rel = ldx(S[0] / np.where(ok, np.abs(Pm), 1.0), S[1] - eP) + ldx(dS[0] / np.where(ok, np.abs(Dm), 1.0), dS[1] - eD)
    re, im, e = _xc64_complex(inc.cpu().numpy())
    got_m = ldx(re, e - qe) + 1j * ldx(im, e - qe)
    assert np.all((np.abs(got_m - qm) <= 2.0 ** -49 * np.abs(qm) * rel)[ok])
    # z_next = z - inc where the increment is representable
    q = ldx(qm.real, qe) + 1j * ldx(qm.imag, qe)
    zn = znr.cpu().numpy() + 1j * zni.cpu().numpy()
    z = pts.re + 1j * pts.im
    fin = ok & np.isfinite(q) & (np.abs(q) < 1e300)
    got_q = ldx(re, e) + 1j * ldx(im, e)
    assert np.all(np.abs(zn - (z - got_q))[fin] <= 4e-16 * (np.abs(z) + np.abs(got_q))[fin])
    # dL/dz = g conj(P') where P' fits FP64
    gc = g[0] + 1j * g[1]
    Dv = ldx(Dm.real, eD) + 1j * ldx(Dm.imag, eD)
    dSv = ldx(dS[0], dS[1])
    rep = ok & (np.abs(Dv) < 1e280) & (dSv < 1e280)
    gz = gz_re.cpu().numpy() + 1j * gz_im.cpu().numpy()
    assert np.all((np.abs(gz - gc * np.conj(Dv)) <= 2.0 ** -49 * np.abs(gc) * dSv)[rep])
    assert rep.sum() > 1000


def _dense_coeff_grad(z, g, n_coef):
    """sum_j g_j conj(z_j)^k for every k, by a running power (FP64)."""
    w = np.ones_like(z)
    cz = np.conj(z)
    G = np.zeros(n_coef, dtype=complex)
    A = np.zeros(n_coef)
    for k in range(n_coef):
        G[k] = np.sum(g * w)
        A[k] = np.sum(np.abs(g) * np.abs(w))
        w = w * cz
    return G, A


def _oracle_windows(coef, zre, zim, l_gpu=None, r_gpu=None):
    """Each point's window [l, r] and G_p from the oracle (p = 53); z = 0 gets the
    window {0} (P(0) = a_0).  When the GPU's windows are given they must be the
    oracle's exactly (a point within 2^-30 of a boundary tie would take either)."""
    pre = oracle.precondition(coef, 53)
    lam = oracle.log2_abs(zre, zim)
    _, _, L, R = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    zero = ~np.isfinite(lam)
    L[zero], R[zero] = 0, 0
    if l_gpu is not None:
        fin = ~zero
        assert np.array_equal(l_gpu[fin], L[fin]) and np.array_equal(r_gpu[fin], R[fin]), \
            "GPU windows differ from the oracle's"
    return L, R, pre.good


def _dense_coeff_grad_windowed(z, g, n_coef, L, R, good):
    """sum_j g_j conj(z_j)^k over each point's kept terms only (L_j <= k <= R_j, k good)."""
    w = np.ones_like(z)
    cz = np.conj(z)
    G = np.zeros(n_coef, dtype=complex)
    A = np.zeros(n_coef)
    for k in range(n_coef):
        m = (L <= k) & (k <= R) & bool(good[k])
        G[k] = np.sum((g * w)[m])
        A[k] = np.sum((np.abs(g) * np.abs(w))[m])
        w = w * cz
    return G, A


@pytest.mark.parametrize("long_window", [4096, 32], ids=["short-windows", "long-windows"])
def test_coefficient_gradient_vs_dense(env, long_window):
    """dL/da_k restricted to the kept terms equals the windowed dense sum; against
    the full (unrestricted) gradient the difference, scaled by |a_k|, is below
    2^(-T+1) sum_j |g_j| M_j (every dropped term is below 2^(-T+1) M_j, §6).
    With the long-window threshold at 32 every window goes through the
    warp-per-point kernel instead of the shared-memory tiles."""
    torch, F = env
    rng = np.random.default_rng(22)
    coef = W.unit_disk_complex(300, rng)
    r = rng.uniform(0.5, 1.3, 800)
    t = rng.uniform(0, 2 * math.pi, 800)
    z = r * np.exp(1j * t)
    g = rng.normal(size=800) + 1j * rng.normal(size=800)
    P = F.fpe_precondition(coef.re, coef.im, None, 53, F.FPE_WITH_DERIV)
    F.fpe_set_tuning(P, long_window, 1024)
    zr = torch.from_numpy(z.real.copy()).cuda()
    zi = torch.from_numpy(z.imag.copy()).cuda()
    ga_re = torch.zeros(coef.n_coef, dtype=torch.float64, device="cuda")
    ga_im = torch.zeros_like(ga_re)
    F.fpe_grad_coeffs(P, zr, zi, torch.from_numpy(g.real.copy()).cuda(), torch.from_numpy(g.imag.copy()).cuda(),
                      ga_re, ga_im)
    F.fpe_eval(P, zr, zi)
    l, rr, _ = F.fpe_get_windows(P, z.size)
    F.fpe_sync(P)
    got = ga_re.cpu().numpy() + 1j * ga_im.cpu().numpy()
    L, R, good = _oracle_windows(coef, z.real.copy(), z.imag.copy(), l.cpu().numpy(), rr.cpu().numpy())
    Gw, Aw = _dense_coeff_grad_windowed(z, g, coef.n_coef, L, R, good)
    assert np.all(np.abs(got - Gw) <= 1e-12 * Aw + 1e-300)
    G, A = _dense_coeff_grad(z, g, coef.n_coef)
    _, _, l2M = oracle.horner_ref(coef, z.real.copy(), z.imag.copy())
    T = F.fpe_info(P)["T"]
    bound = 2.0 ** (-T + 1) * np.sum(np.abs(g) * np.exp2(l2M))
    a_abs = np.hypot(coef.re, coef.im)
    assert np.all(a_abs * np.abs(got - G) <= bound + 1e-12 * a_abs * A)


@pytest.mark.parametrize("long_window", [4096, 32], ids=["short-windows", "long-windows"])
def test_coefficient_gradient_real(env, long_window):
    """Real coefficients at real points (ga_im NULL), including z = 0 (only
    a_0 moves P(0)) and a warp mixing |z| far apart (the per-point fallback)."""
    torch, F = env
    rng = np.random.default_rng(24)
    coef = W.Coeffs(rng.uniform(-1, 1, 401), None)
    x = np.concatenate([rng.uniform(-1.2, 1.2, 700), [0.0], [1e-30, 3e20], rng.uniform(-1.05, 1.05, 97)])
    g = rng.normal(size=x.size)
    P = F.fpe_precondition(coef.re, None, None, 53)
    F.fpe_set_tuning(P, long_window, 1024)
    xr = torch.from_numpy(x.copy()).cuda()
    ga = torch.zeros(coef.n_coef, dtype=torch.float64, device="cuda")
    F.fpe_grad_coeffs(P, xr, None, torch.from_numpy(g.copy()).cuda(), None, ga, None)
    F.fpe_eval(P, xr, None)
    l, rr, _ = F.fpe_get_windows(P, x.size)
    F.fpe_sync(P)
    # the oracle's windows (z = 0: the window {0}, as P(0) = a_0)
    L, R, good = _oracle_windows(coef, x.copy(), None, l.cpu().numpy(), rr.cpu().numpy())
    with np.errstate(over="ignore", invalid="ignore"):
        Gw, Aw = _dense_coeff_grad_windowed(x.astype(complex), g.astype(complex), coef.n_coef, L, R, good)
    got = ga.cpu().numpy()
    fin = np.isfinite(Gw.real)
    assert np.all((np.abs(got - Gw.real) <= 1e-12 * Aw + 1e-300)[fin])


def test_autograd_finite_differences(env):
    """loss = sum |P(z_j) - t_j|^2; autograd's gradients against central
    differences with h = 1e-6."""
    torch, F = env
    from paper_2211_06320_gb300.autograd import poly_eval, precondition_for_grad
    rng = np.random.default_rng(23)
    d, n = 200, 300
    coef = W.unit_disk_complex(d, rng)
    a = torch.tensor(coef.re + 1j * coef.im, dtype=torch.complex128, device="cuda", requires_grad=True)
    rr = rng.uniform(0.3, 1.0, n)
    tt = rng.uniform(0, 2 * math.pi, n)
    z = torch.tensor(rr * np.exp(1j * tt), dtype=torch.complex128, device="cuda", requires_grad=True)
    tgt = torch.tensor(rng.normal(size=n) + 1j * rng.normal(size=n), dtype=torch.complex128, device="cuda")

    def loss_of(av, zv):
        with torch.no_grad():
            poly = precondition_for_grad(av)
            y = poly_eval(av, zv, poly)
            return float(torch.sum(torch.abs(y - tgt) ** 2).item())

    poly = precondition_for_grad(a)
    y = poly_eval(a, z, poly)
    L = torch.sum(torch.abs(y - tgt) ** 2)
    L.backward()
    h = 1e-6
    for k in (0, 1, 57, 199):
        for unit in (1.0, 1j):
            ap, am = a.detach().clone(), a.detach().clone()
            ap[k] += h * unit
            am[k] -= h * unit
            fd = (loss_of(ap, z.detach()) - loss_of(am, z.detach())) / (2 * h)
            gk = a.grad[k].item()
            an = gk.real if unit == 1.0 else gk.imag
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, unit, fd, an)
    for j in (0, 7, 150, 299):
        for unit in (1.0, 1j):
            zp, zm = z.detach().clone(), z.detach().clone()
            zp[j] += h * unit
            zm[j] -= h * unit
            fd = (loss_of(a.detach(), zp) - loss_of(a.detach(), zm)) / (2 * h)
            gj = z.grad[j].item()
            an = gj.real if unit == 1.0 else gj.imag
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (j, unit, fd, an)


def test_differentiation_workload_reduced(env):
    """The differentiation workload's shape at d = 2^14, 2^14 points with |z| <= 1:
    forward P, Newton step, and dL/da_k against the dense gradient."""
    torch, F = env
    from paper_2211_06320_gb300.autograd import poly_eval, precondition_for_grad
    wl, a_true, tn = W.differentiation_d2pow18(n_points=1 << 15, d=1 << 14)
    z = wl.points.re + 1j * wl.points.im
    keep = np.abs(z) <= 1.0
    z = z[keep][:1 << 14]
    at = a_true.re + 1j * a_true.im
    # targets from the true polynomial, evaluated by the oracle
    ref_t, _, _ = oracle.horner_ref(a_true, z.real.copy(), z.imag.copy())
    t = (ref_t.re_hi + ref_t.re_lo) * 2.0 ** ref_t.e + 1j * (ref_t.im_hi + ref_t.im_lo) * 2.0 ** ref_t.e
    t = t + (tn[keep][:1 << 14, 0] + 1j * tn[keep][:1 << 14, 1])
    a = torch.tensor(wl.coeffs.re + 1j * wl.coeffs.im, dtype=torch.complex128, device="cuda", requires_grad=True)
    zt = torch.tensor(z, dtype=torch.complex128, device="cuda")
    tt = torch.tensor(t, dtype=torch.complex128, device="cuda")
    poly = precondition_for_grad(a)
    y = poly_eval(a, zt, poly)
    L = torch.sum(torch.abs(y - tt) ** 2)
    L.backward()
    # dense reference: g = 2 (P - t) (PyTorch's gradient of |.|^2), grad_a = sum g conj(z)^k
    ref, S, _ = oracle.horner_ref(wl.coeffs, z.real.copy(), z.imag.copy())
    Pv = (ref.re_hi + ref.re_lo) * 2.0 ** ref.e + 1j * (ref.im_hi + ref.im_lo) * 2.0 ** ref.e
    g = 2 * (Pv - t)
    F.fpe_eval(poly, zt.real.contiguous(), zt.imag.contiguous())
    l, rr, _ = F.fpe_get_windows(poly, z.size)
    L, R, good = _oracle_windows(wl.coeffs, z.real.copy(), z.imag.copy(), l.cpu().numpy(), rr.cpu().numpy())
    G, A = _dense_coeff_grad_windowed(z, g, wl.coeffs.n_coef, L, R, good)
    got = a.grad.detach().cpu().numpy()
    assert np.all(np.abs(got - G) <= 1e-10 * A + 1e-300)
    inc, _, _ = F.fpe_newton(poly, zt.real.contiguous(), zt.imag.contiguous())
    F.fpe_sync(poly)
    assert np.all(np.isfinite(inc.cpu().numpy()[:, :2]))
