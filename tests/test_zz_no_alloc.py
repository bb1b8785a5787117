"""fpe_eval_noalloc: evaluation for callers that cannot allocate device memory
while they evaluate (a fixed device-memory budget set at start-up, a
latency-bound loop that must not pay for cudaMalloc and the synchronisation it
implies, a host that hands the library only buffers it owns).  Its scratch is
one built-in array in the library's device memory, shared by every call.

Checked here, through the C ABI, on two calls in a row (so stale contents of
the shared array from the first call would show in the second):
  * the values against the CPU oracle's window sums on the oracle's own
    windows, within the parity tolerance (2^-50 S_w for p = 53, 2^-21 S_w for
    p = 24 in FP32 mode);
  * the values, kept-term counts and cancelled-bit estimates against fpe_eval
    on the same handle (tensor-core path off, so both run the same kernels);
  * every mode: the default FP64 summation, FPE_FP32, FPE_ACCURATE, real
    coefficients, real and complex points;
  * z = 0 and a NaN point (status FPE_ERR_NONFINITE from the next fpe_sync);
  * no device allocation: free device memory is unchanged across calls.
This file is collected last so that a failure here leaves every other test
already run."""
import math

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


def _against_oracle(coef, p, zre, zim, out, nt, l_gpu, r_gpu, tol):
    pre = oracle.precondition(coef, p)
    lam = oracle.log2_abs(zre, zim)
    kl, No, Lo, Ro = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    fin = np.isfinite(lam)
    agree = windows_agree(l_gpu[fin], r_gpu[fin], Lo[fin], Ro[fin], pre.hk, pre.hs, pre.T, lam[fin], No[fin])
    assert agree.all(), f"{(~agree).sum()} windows differ from the oracle's beyond boundary ties"
    L2, R2 = Lo.copy(), Ro.copy()
    L2[~fin], R2[~fin] = 0, 0
    Q, SQ = oracle.window_sum(coef, pre.good, zre, zim, L2, R2, with_S=True)
    r = error_ratio(out[fin], oracle.ExtValues(np.stack([Q.re_hi, Q.re_lo, Q.im_hi, Q.im_lo], 1)[fin], Q.e[fin]),
                    (SQ[0][fin], SQ[1][fin]), tol * 31 / 32)
    assert r.max() <= 1.0, f"noalloc differs from the oracle's window sum by {r.max():.3g} x tolerance"
    # kept-term counts where the windows are the oracle's exactly
    cg = np.concatenate([[0], np.cumsum(pre.good)])
    want_nt = cg[np.minimum(Ro, pre.d) + 1] - cg[Lo]
    same = fin.copy()
    same[fin] = (l_gpu[fin] == Lo[fin]) & (r_gpu[fin] == Ro[fin])
    assert np.array_equal(nt[same], want_nt[same])
    return r.max()


def _call_pair(env, P, coef, p, zre, zim, tol):
    torch, F = env
    n = zre.shape[0]
    zr = torch.from_numpy(np.ascontiguousarray(zre)).cuda()
    zi = None if zim is None else torch.from_numpy(np.ascontiguousarray(zim)).cuda()
    outs = [F.empty_out(n) for _ in range(2)]
    nts = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(2)]
    bls = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(2)]
    # the first call on a device may load the library's device code (and with
    # it the built-in array); free memory is compared across the call after it
    F.fpe_eval_noalloc(P, zr, zi, outs[0], nts[0], bls[0])
    F.fpe_sync(P)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    F.fpe_eval_noalloc(P, zr, zi, outs[0], nts[0], bls[0])
    F.fpe_sync(P)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"fpe_eval_noalloc changed free device memory by {free0 - free1} bytes"
    F.fpe_set_tensor_path(P, 0)  # fpe_eval on the same FP64 kernels
    F.fpe_eval(P, zr, zi, outs[1], nts[1], bls[1])
    l, rr, _ = F.fpe_get_windows(P, n)  # the windows of the locate kernel both calls share
    F.fpe_sync(P)
    a, b = outs[0].cpu().numpy(), outs[1].cpu().numpy()
    nta, ntb = nts[0].cpu().numpy(), nts[1].cpu().numpy()
    assert np.array_equal(nta, ntb), "kept-term counts differ from fpe_eval"
    assert np.array_equal(bls[0].cpu().numpy(), bls[1].cpu().numpy()), "cancelled-bit estimates differ from fpe_eval"
    # against fpe_eval's output, in the oracle's tolerance scale S(z)
    _, S, _ = oracle.horner_ref(coef, zre, zim)
    be = np.ascontiguousarray(b[:, 2]).view(np.int64)
    ref = oracle.ExtValues(np.stack([b[:, 0], np.zeros(n), b[:, 1], np.zeros(n)], axis=1), be)
    r = error_ratio(a, ref, S, tol)
    assert r.max() <= 1.0, f"noalloc differs from fpe_eval by {r.max():.3g} x tolerance"
    return _against_oracle(coef, p, zre, zim, a, nta, l.cpu().numpy(), rr.cpu().numpy(), tol)


MODES = {"fp64": (53, 0), "fp32": (24, 4), "accurate": (53, 16)}


@pytest.mark.parametrize("points", ["complex", "real"])
@pytest.mark.parametrize("coefs", ["complex", "real"])
@pytest.mark.parametrize("mode", list(MODES))
def test_noalloc_matches_oracle_and_fpe_eval_twice(env, mode, coefs, points):
    torch, F = env
    p, flags = MODES[mode]
    rng = np.random.default_rng(2468 + 7 * len(mode) + (coefs == "real") * 3 + (points == "real"))
    c = W.unit_disk_complex(6000, rng)
    coef = W.Coeffs(c.re, None) if coefs == "real" else c
    if coefs == "real":
        flags |= F.FPE_REAL
    P = F.fpe_precondition(coef.re, coef.im, None, p, flags)
    tol = TOL_FP32 if p == 24 else TOL_FP64
    # first call: as many points as the built-in scratch takes (short windows and some long ones)
    if points == "complex":
        p1 = W.sphere_points(F.NOALLOC_MAX_POINTS, rng)
        zr1, zi1 = p1.re, p1.im
    else:
        zr1, zi1 = rng.uniform(-2.0, 2.0, F.NOALLOC_MAX_POINTS), None
    _call_pair(env, P, coef, p, zr1, zi1, tol)
    # second call on other points: |z| = 1, every window long (warp groups), so
    # contents left in the shared array by the first call would show
    m = 3000
    if points == "complex":
        t = rng.uniform(0, 2 * math.pi, m)
        zr2, zi2 = np.cos(t), np.sin(t)
    else:
        zr2, zi2 = np.where(rng.uniform(size=m) < 0.5, -1.0, 1.0) * rng.uniform(0.999, 1.001, m), None
    _call_pair(env, P, coef, p, zr2, zi2, tol)


def test_noalloc_zero_and_nonfinite_points(env):
    """z = 0 gives a_0, a NaN point gives NaN and FPE_ERR_NONFINITE at fpe_sync,
    and the next call on finite points is clean."""
    torch, F = env
    rng = np.random.default_rng(11)
    coef = W.unit_square_complex(200, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    zr = torch.tensor([0.0, 0.5, float("nan"), -0.25], dtype=torch.float64, device="cuda")
    zi = torch.tensor([0.0, 0.5, 0.0, 0.75], dtype=torch.float64, device="cuda")
    out = F.fpe_eval_noalloc(P, zr, zi)
    with pytest.raises(F.FpeError) as e:
        F.fpe_sync(P)
    assert e.value.status == F.FPE_ERR_NONFINITE
    o = out.cpu().numpy()
    e0 = int(np.ascontiguousarray(o[:, 2]).view(np.int64)[0])
    assert math.ldexp(o[0, 0], e0) == coef.re[0] and math.ldexp(o[0, 1], e0) == coef.im[0]
    assert np.isnan(o[2, 0]) and np.isnan(o[2, 1])
    F.fpe_eval_noalloc(P, zr[[0, 1, 3]].contiguous(), zi[[0, 1, 3]].contiguous())
    F.fpe_sync(P)  # no status left over from the previous call


def test_noalloc_rejects_too_many_points(env):
    torch, F = env
    coef = W.unit_square_complex(50, np.random.default_rng(1))
    P = F.fpe_precondition(coef.re, coef.im)
    z = torch.zeros(F.NOALLOC_MAX_POINTS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FpeError) as e:
        F.fpe_eval_noalloc(P, z, z)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
