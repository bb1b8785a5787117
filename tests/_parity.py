"""Comparison helpers for the parity tests (test infrastructure)."""
import numpy as np

TOL_FP64 = 2.0 ** -50   # |P_gpu - P_ref| <= 2^-50 S(z) for p = 53
TOL_FP32 = 2.0 ** -21   # and 2^-21 S(z) for p = 24


def _scaled(m, e, ref_e):
    sh = np.clip(e - ref_e, -2000, 2000).astype(np.int64)
    return np.ldexp(m, sh.astype(np.int32))


def error_ratio(gpu_out: np.ndarray, ref, S, tol: float = TOL_FP64) -> np.ndarray:
    """|gpu - ref| / (tol * S) per point, all in S's exponent frame.

    gpu_out: (n, 3) fpe_xc64 rows (re, im, e-bits); ref: oracle.ExtValues;
    S: (mantissa, exponent) arrays.  Points with S = 0 compare exactly."""
    g_re, g_im = gpu_out[:, 0], gpu_out[:, 1]
    g_e = np.ascontiguousarray(gpu_out[:, 2]).view(np.int64)
    Sm, Se = S
    fr = _scaled(g_re, g_e, Se) - (_scaled(ref.re_hi, ref.e, Se) + _scaled(ref.re_lo, ref.e, Se))
    fi = _scaled(g_im, g_e, Se) - (_scaled(ref.im_hi, ref.e, Se) + _scaled(ref.im_lo, ref.e, Se))
    err = np.hypot(fr, fi)
    denom = tol * Sm
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(denom > 0, err / denom, np.where(err == 0, 0.0, np.inf))
    r[~np.isfinite(g_re) | ~np.isfinite(g_im)] = np.inf
    return r


def xc64_to_complex_scaled(gpu_out: np.ndarray, ref_e: np.ndarray):
    g_e = np.ascontiguousarray(gpu_out[:, 2]).view(np.int64)
    return _scaled(gpu_out[:, 0], g_e, ref_e) + 1j * _scaled(gpu_out[:, 1], g_e, ref_e)


def windows_agree(l_gpu, r_gpu, l_ref, r_ref, hk, hs, T, lam, N) -> np.ndarray:
    """Per point: windows equal, or differ only at a boundary k whose
    cover(k) + lambda k is within 2^-30 max(1, |N|) of the threshold N - T
    (either decision is correct there)."""
    from fractions import Fraction
    import oracle
    ok = (l_gpu == l_ref) & (r_gpu == r_ref)
    for j in np.nonzero(~ok)[0]:
        good = True
        thr = float(N[j]) - T
        tol = 2.0 ** -30 * max(1.0, abs(float(N[j])))
        # k kept by one side only: [min l, max l - 1] on the left, [min r + 1, max r] on the right
        diff = list(range(min(l_gpu[j], l_ref[j]), max(l_gpu[j], l_ref[j])))
        diff += list(range(min(r_gpu[j], r_ref[j]) + 1, max(r_gpu[j], r_ref[j]) + 1))
        if len(diff) > 4:
            good = False
        else:
            for k in diff:
                if not (hk[0] <= k <= hk[-1]):
                    good = False
                    break
                v = float(oracle.cover_value(hk, hs, int(k))) + float(lam[j]) * k
                if abs(v - thr) > tol:
                    good = False
        ok[j] = good
    return ok
