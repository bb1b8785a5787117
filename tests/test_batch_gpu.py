"""Batched evaluation (many polynomials, one fixed launch sequence) against
the oracle, in FP64 and FP32, and replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TOL_FP32, TOL_FP64, error_ratio

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_06320_gb300 as F
    F._load()
    return torch, F


def _batch_inputs(n_poly, pts_per_poly, seed, dmax=1 << 16):
    wls = W.batched_lognormal(n_poly=n_poly, pts_per_poly=pts_per_poly, seed=seed, dmax=dmax)
    offs = np.concatenate([[0], np.cumsum([w.points.n for w in wls])]).astype(np.int64)
    zre = np.concatenate([w.points.re for w in wls])
    zim = np.concatenate([w.points.im for w in wls])
    return wls, offs, zre, zim


def _check_against_oracle(wls, offs, out, nt, p, tol, sample):
    for i in sample:
        w = wls[i]
        pre = oracle.precondition(w.coeffs, p)
        sl = slice(offs[i], offs[i + 1])
        vals, (kl, N, L, R) = oracle.fpe_eval(pre, w.points.re, w.points.im, with_S=True)
        Q, SQ = vals
        r = error_ratio(out[sl], Q, SQ, tol * 31 / 32)
        assert r.max() <= 1.0, f"polynomial {i}: {r.max():.3g} x tolerance"
        cg = np.concatenate([[0], np.cumsum(pre.good)])
        want = cg[R + 1] - cg[L]
        # kept-term counts agree except where a window boundary is a near tie
        assert np.mean(nt[sl] == want) > 0.99


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_batch_lognormal(env, fp32):
    """Config-4 shape: log-uniform degrees in [16, 2^16], log2|a_k| = s k + N(0,4),
    256 sphere points each (512 polynomials here; a sample checked by the oracle)."""
    torch, F = env
    wls, offs, zre, zim = _batch_inputs(512, 256, seed=3)
    p = 24 if fp32 else 53
    flags = F.FPE_FP32 if fp32 else 0
    polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im, None, p, flags) for w in wls]
    B = F.fpe_batch_create(polys, offs)
    zr = torch.from_numpy(zre).cuda()
    zi = torch.from_numpy(zim).cuda()
    nt = torch.empty(B.n, dtype=torch.int32, device="cuda")
    out = F.fpe_batch_eval(B, zr, zi, nterms=nt)
    F.fpe_batch_sync(B)
    out, nt = out.cpu().numpy(), nt.cpu().numpy()
    degs = np.array([w.coeffs.n_coef for w in wls])
    sample = sorted(set(np.argsort(-degs)[:6].tolist()) | set(range(0, 512, 16)))
    _check_against_oracle(wls, offs, out, nt, p, TOL_FP32 if fp32 else TOL_FP64, sample)


def test_batch_equals_single_handles(env):
    torch, F = env
    wls, offs, zre, zim = _batch_inputs(40, 300, seed=5, dmax=20000)
    polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im) for w in wls]
    B = F.fpe_batch_create(polys, offs)
    zr = torch.from_numpy(zre).cuda()
    zi = torch.from_numpy(zim).cuda()
    out = F.fpe_batch_eval(B, zr, zi).cpu().numpy()
    for i, P in enumerate(polys):
        sl = slice(offs[i], offs[i + 1])
        # a batch sums every window with the FP64 window kernels; so does a single
        # handle with the tensor-core path off, bit for bit
        F.fpe_set_tensor_path(P, 0)
        single = F.fpe_eval(P, zr[sl].contiguous(), zi[sl].contiguous()).cpu().numpy()
        assert np.array_equal(single.view(np.int64), out[sl].view(np.int64)), i


def test_batch_graph_capture_replay(env):
    """fpe_batch_eval allocates nothing and never synchronises, so it can be
    captured in a CUDA graph and replayed on new points."""
    torch, F = env
    wls, offs, zre, zim = _batch_inputs(64, 256, seed=7, dmax=30000)
    polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im) for w in wls]
    B = F.fpe_batch_create(polys, offs)
    zr = torch.from_numpy(zre).cuda()
    zi = torch.from_numpy(zim).cuda()
    out = F.empty_out(B.n)
    F.fpe_batch_eval(B, zr, zi, out=out)  # warm-up outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        F.fpe_batch_eval(B, zr, zi, out=out, stream=s)
    rng = np.random.default_rng(99)
    for _ in range(2):
        pts = W.sphere_points(B.n, rng)
        zr.copy_(torch.from_numpy(pts.re))
        zi.copy_(torch.from_numpy(pts.im))
        g.replay()
        torch.cuda.synchronize()
        want = F.fpe_batch_eval(B, zr, zi).cpu().numpy()
        assert np.array_equal(out.cpu().numpy().view(np.int64), want.view(np.int64))


def test_batch_rejects_mixed_modes(env):
    torch, F = env
    a = W.unit_square_complex(50, np.random.default_rng(1))
    p1 = F.fpe_precondition(a.re, a.im)
    p2 = F.fpe_precondition(a.re, None)
    with pytest.raises(F.FpeError) as e:
        F.fpe_batch_create([p1, p2], [0, 10, 20])
    assert e.value.status == F.FPE_ERR_UNSUPPORTED
    p3 = F.fpe_precondition(a.re, a.im, None, 24, F.FPE_FP32)
    with pytest.raises(F.FpeError):
        F.fpe_batch_create([p1, p3], [0, 10, 20])


def test_batch_empty_segments(env):
    torch, F = env
    rng = np.random.default_rng(11)
    coefs = [W.unit_square_complex(d, rng) for d in (5, 300, 2000)]
    polys = [F.fpe_precondition(c.re, c.im) for c in coefs]
    offs = np.array([0, 0, 100, 100], dtype=np.int64)
    pts = W.sphere_points(100, rng)
    B = F.fpe_batch_create(polys, offs)
    out = F.fpe_batch_eval(B, torch.from_numpy(pts.re).cuda(), torch.from_numpy(pts.im).cuda()).cpu().numpy()
    F.fpe_batch_sync(B)
    ref, S, _ = oracle.horner_ref(coefs[1], pts.re, pts.im)
    assert error_ratio(out, ref, S).max() <= 1.0
