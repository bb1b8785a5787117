"""The C-ABI library builds, loads and exports every symbol include/fpe.h
declares; its host preconditioning (scales, concave cover, G_p) is bit-exact
against the oracle; argument errors are reported.  No GPU needed: these use
FPE_HOST_ONLY handles, which touch no device memory."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    import paper_2211_06320_gb300 as F
    F._load()
    return F


def test_header_symbols_exported(F):
    hdr = open(os.path.join(ROOT, "include", "fpe.h")).read() + open(os.path.join(ROOT, "include", "fpe_bench.h")).read()
    # function declarations: a return type at the start of a line, then the name
    declared = set(re.findall(r"^(?:fpe_status|void|const char \*)\s*(fpe_[a-z_0-9]+)\s*\(", hdr, re.M))
    assert declared, "no declarations found"
    lib = ctypes.CDLL(F.library_path())
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in fpe.h but not exported"
    assert declared == set(F.EXPORTED)


def _host(F, coef, p=53, flags=0):
    return F.fpe_precondition(coef.re, coef.im, coef.e2, p, flags | F.FPE_HOST_ONLY)


def _families():
    rng = np.random.default_rng(2024)
    out = [
        ("unit_square_1000", W.unit_square_complex(1000, rng)),
        ("unit_disk_65536", W.unit_disk_complex(1 << 16, rng)),
        ("half_circle_1000", W.half_circle(1000)),
        ("half_circle_c_700", W.half_circle(700, True, rng)),
        ("inverse_factorial_5000", W.inverse_factorial(5000)),
        ("mandelbrot_9", W.mandelbrot(9)),
        ("sparse_65536", W.sparse_real(1 << 16, 0.01, rng)),
        ("lognormal_3000", W.lognormal_profile(3000, 0.008, rng)),
        ("chebyshev_120", W.chebyshev_T(120)),
        ("geometric_50", W.geometric(50)),
        ("xpow_minus1_64", W.power_minus_one(64)),
        ("worked_example", W.worked_example_coeffs(rng)),
        ("constant", W.Coeffs(np.array([3.5]))),
        ("one_plus_z", W.Coeffs(np.array([1.0, 1.0]))),
    ]
    # leading and trailing zeros, extended exponents spanning far beyond FP64
    c = W.unit_square_complex(300, rng)
    c.re[:7] = 0.0
    c.im[:7] = 0.0
    c.re[-5:] = 0.0
    c.im[-5:] = 0.0
    out.append(("trimmed_300", c))
    e2 = rng.integers(-100000, 100000, 400)
    out.append(("ext_random_400", W.Coeffs(rng.uniform(-1, 1, 400), rng.uniform(-1, 1, 400), e2)))
    # complex values whose modulus sits exactly on or next to a power of two
    vals = np.array([0.6, 0.8, 3.0, 4.0, 1.0, 0.0, 2.0 ** -30, 1.0 - 2 ** -53])
    out.append(("boundary_moduli", W.Coeffs(vals, vals[::-1].copy())))
    return out


@pytest.mark.parametrize("name,coef", _families(), ids=[n for n, _ in _families()])
def test_host_precondition_bitexact(F, name, coef):
    for p in (53, 24, 6):
        P = _host(F, coef, p)
        pre = oracle.precondition(coef, p)
        info = F.fpe_info(P)
        assert info["d"] == pre.d and info["valuation"] == pre.v and info["T"] == pre.T
        k, s = F.fpe_get_hull(P)
        assert np.array_equal(k, pre.hk) and np.array_equal(s, pre.hs), name
        g = F.fpe_get_good(P)
        assert np.array_equal(g, pre.good), name
        assert info["n_good"] == int(pre.good.sum())


def test_host_scale_single_coefficient(F):
    """A single nonzero coefficient's cover is its scale: s(3+2i)=2, s(3+3i)=3 (§2.3)."""
    for (x, y), want in [((3.0, 2.0), 2), ((3.0, 3.0), 3), ((3.0, 4.0), 3), ((1.0, 0.0), 1), ((0.0, -0.75), 0)]:
        P = F.fpe_precondition(np.array([x]), np.array([y]), None, 53, F.FPE_HOST_ONLY)
        k, s = F.fpe_get_hull(P)
        assert list(s) == [want]


def test_precondition_errors(F):
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.zeros(5), None, None, 53, F.FPE_HOST_ONLY)
    assert e.value.status == F.FPE_ERR_ZERO_POLY
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.array([1.0, np.nan]), None, None, 53, F.FPE_HOST_ONLY)
    assert e.value.status == F.FPE_ERR_NONFINITE
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.array([1.0, 2.0]), np.array([0.0, np.inf]), None, 53, F.FPE_HOST_ONLY)
    assert e.value.status == F.FPE_ERR_NONFINITE
    for p in (0, 1, 54, 100):
        with pytest.raises(F.FpeError) as e:
            F.fpe_precondition(np.array([1.0, 2.0]), None, None, p, F.FPE_HOST_ONLY)
        assert e.value.status == F.FPE_ERR_INVALID_ARG
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.array([1.0, 2.0]), None, None, 53, 1 << 20)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.zeros(0), None, None, 53, F.FPE_HOST_ONLY)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
    with pytest.raises(F.FpeError) as e:
        F.fpe_precondition(np.array([1.0]), None, np.array([1 << 50]), 53, F.FPE_HOST_ONLY)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
    with pytest.raises(F.FpeError) as e:  # the forced window-sum kinds exclude each other
        F.fpe_precondition(np.array([1.0, 2.0]), None, None, 53,
                           F.FPE_HOST_ONLY | F.FPE_FORCE_DENSE | F.FPE_FORCE_SPARSE)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
    for fl in (F.FPE_FORCE_DENSE, F.FPE_FORCE_SPARSE):  # each alone is accepted
        F.fpe_precondition(np.array([1.0, 2.0]), None, None, 53, F.FPE_HOST_ONLY | fl)


def test_host_only_handle_refuses_evaluation(F):
    lib = F._load()
    P = F.fpe_precondition(np.array([1.0, 2.0]), None, None, 53, F.FPE_HOST_ONLY)
    z = np.zeros(4)
    out = np.zeros((4, 3))
    st = lib.fpe_eval(P.handle, F._np_ptr(z), None, 4, F._np_ptr(out), None, None, None)
    assert st == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_sync(P.handle, None) == F.FPE_ERR_INVALID_ARG


def test_null_handle_and_status_strings(F):
    lib = F._load()
    assert lib.fpe_eval(None, None, None, 0, None, None, None, None) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_info(None, None, None, None, None, None) == F.FPE_ERR_INVALID_ARG
    lib.fpe_destroy(None)
    for s in range(8):
        assert F.fpe_status_string(s)


def test_tuning_set_get_and_limits(F):
    """Launch parameters of the window sums: defaults, a valid setting kept,
    out-of-range settings and NULL arguments refused; the autotuner refuses a
    host-only handle before touching any device memory."""
    lib = F._load()
    P = F.fpe_precondition(np.array([1.0, 2.0, 3.0]), None, None, 53, F.FPE_HOST_ONLY)
    assert F.fpe_get_tuning(P) == {"long_window": 4096, "lane_chunk": 1024, "ms": 0.0}
    F.fpe_set_tuning(P, 2048, 256)
    assert F.fpe_get_tuning(P) == {"long_window": 2048, "lane_chunk": 256, "ms": 0.0}
    for lw, lc in [(31, 256), (1 << 25, 256), (4096, 15), (4096, 1 << 17)]:
        with pytest.raises(F.FpeError) as e:
            F.fpe_set_tuning(P, lw, lc)
        assert e.value.status == F.FPE_ERR_INVALID_ARG
    assert F.fpe_get_tuning(P)["long_window"] == 2048
    t = F.Tuning()
    assert lib.fpe_set_tuning(None, ctypes.byref(t)) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_set_tuning(P.handle, None) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_get_tuning(P.handle, None) == F.FPE_ERR_INVALID_ARG
    z = np.zeros(4)
    assert lib.fpe_autotune(P.handle, F._np_ptr(z), None, 4, None, ctypes.byref(t)) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_batch_set_tuning(None, ctypes.byref(t)) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_batch_autotune(None, None, None, None, ctypes.byref(t)) == F.FPE_ERR_INVALID_ARG


def test_derivative_handle_host(F):
    """P' coefficients (k+1) a_{k+1} are preconditioned separately (§7.2)."""
    c = W.unit_square_complex(200, np.random.default_rng(9))
    P = F.fpe_precondition(c.re, c.im, None, 53, F.FPE_HOST_ONLY | F.FPE_WITH_DERIV)
    assert F.fpe_info(P)["d"] == 200


@pytest.mark.parametrize("family", ["half_circle", "lognormal", "worked"])
def test_analyse_intervals_match_oracle_windows(F, family):
    """fpe_analyse: coefficient k is kept at lambda exactly when
    lam_lo[k] <= lambda <= lam_hi[k]; checked against the oracle's windows on a
    grid of lambda (away from the endpoints, where FP64 ties may differ)."""
    rng = np.random.default_rng(3)
    if family == "half_circle":
        coef = W.half_circle(300)
    elif family == "lognormal":
        coef = W.lognormal_profile(400, 0.02, rng)
    else:
        coef = W.worked_example_coeffs(rng)
    p = 12
    P = F.fpe_precondition(coef.re, coef.im, coef.e2, p, F.FPE_HOST_ONLY)
    lo, hi = F.fpe_analyse(P)
    pre = oracle.precondition(coef, p)
    lam = np.linspace(-40, 40, 801) + 0.0137
    kl, N, L, R = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    k = np.arange(coef.n_coef)
    for i, lm in enumerate(lam):
        kept = (k >= L[i]) & (k <= R[i]) & pre.good.astype(bool)
        pred = (lo <= lm) & (lm <= hi)
        clear = np.isnan(lo) | ((np.abs(lm - lo) > 1e-9) & (np.abs(lm - hi) > 1e-9))
        assert np.array_equal(kept[clear], pred[clear]), (family, lm)
    assert np.all(np.isnan(lo) == ~pre.good.astype(bool))


def test_tensor_path_settings_host(F):
    """The tensor-core threshold of a handle: 384 by default; 0 (off) and
    [32, 2^30] accepted, anything else and a NULL handle refused without
    changing the setting.  A flat cover is one long piece that qualifies;
    FPE_FP32 and FPE_ACCURATE handles qualify none (those modes never take
    the path)."""
    lib = F._load()
    c = W.unit_disk_complex(4096, np.random.default_rng(11))
    for k in (0, 4096):  # |a_0| = |a_d| = 0.9: the largest scale at both ends, one flat piece
        r = float(np.hypot(c.re[k], c.im[k])) or 1.0
        c.re[k], c.im[k] = 0.9 * c.re[k] / r, 0.9 * c.im[k] / r
    P = F.fpe_precondition(c.re, c.im, None, 53, F.FPE_HOST_ONLY)
    assert F.fpe_get_tensor_path(P) == {"min_window": 384, "pieces": 1}
    for mw in (0, 32, 1000, 1 << 30):
        F.fpe_set_tensor_path(P, mw)
        assert F.fpe_get_tensor_path(P)["min_window"] == mw
    for mw in (-1, 1, 31, (1 << 30) + 1):
        with pytest.raises(F.FpeError) as e:
            F.fpe_set_tensor_path(P, mw)
        assert e.value.status == F.FPE_ERR_INVALID_ARG
    assert F.fpe_get_tensor_path(P)["min_window"] == 1 << 30
    assert lib.fpe_set_tensor_path(None, 384) == F.FPE_ERR_INVALID_ARG
    assert lib.fpe_get_tensor_path(None, None, None) == F.FPE_ERR_INVALID_ARG
    for flag, p in ((F.FPE_FP32, 24), (F.FPE_ACCURATE, 53)):
        Q = F.fpe_precondition(c.re, c.im, None, p, F.FPE_HOST_ONLY | flag)
        assert F.fpe_get_tensor_path(Q)["pieces"] == 0
