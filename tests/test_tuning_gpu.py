"""Launch parameters of the window sums (long-window threshold, lane chunk)
and the autotuner: every setting schedules the same kept terms, so values stay
within the tolerance against the oracle's window sums; the autotuner returns a
setting of its grid and keeps it in the handle (or batch)."""
import numpy as np
import pytest

import oracle
import workloads as W
from _parity import TOL_FP64, error_ratio

pytestmark = pytest.mark.gpu

GRID_LW = {1024, 2048, 4096, 8192}
GRID_LC = {128, 256, 512, 1024, 2048}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_06320_gb300 as F
    F._load()
    return torch, F


def _near_unit_circle(n, rng):
    """Points with |z| within 2^-8 of 1 (long windows), random phases."""
    lam = rng.uniform(-2.0 ** -8, 2.0 ** -8, n)
    th = rng.uniform(0, 2 * np.pi, n)
    r = 2.0 ** lam
    return W.Points(r * np.cos(th), r * np.sin(th))


def _check(env, P, coef, pts, sample=None):
    torch, F = env
    zr = torch.from_numpy(pts.re).cuda()
    zi = None if pts.im is None else torch.from_numpy(pts.im).cuda()
    out = F.fpe_eval(P, zr, zi).cpu().numpy()
    F.fpe_sync(P)
    pre = oracle.precondition(coef, 53)
    idx = np.arange(pts.n) if sample is None else sample
    lam = oracle.log2_abs(pts.re[idx], None if pts.im is None else pts.im[idx])
    _, _, Lo, Ro = oracle.windows(pre.hk, pre.hs, pre.T, lam)
    Q, SQ = oracle.window_sum(coef, pre.good, pts.re[idx], None if pts.im is None else pts.im[idx], Lo, Ro,
                              with_S=True)
    r = error_ratio(out[idx], Q, SQ, TOL_FP64 * 31 / 32)
    assert r.max() <= 1.0, f"{r.max():.3g} x tolerance"
    return float(r.max())


@pytest.mark.parametrize("lw,lc", [(32, 16), (64, 37), (1024, 256), (1 << 24, 1024)],
                         ids=["lw32-lc16", "lw64-lc37", "lw1024-lc256", "all-per-thread"])
def test_settings_keep_parity(env, lw, lc):
    """Extreme settings: every window of more than 32 terms in groups of
    16-term lane chunks (hundreds of groups per window), an odd chunk length,
    and no groups at all; windows up to ~2^14 terms near |z| = 1."""
    torch, F = env
    rng = np.random.default_rng(31)
    coef = W.unit_disk_complex(1 << 14, rng)
    pts = _near_unit_circle(1500, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    F.fpe_set_tuning(P, lw, lc)
    assert F.fpe_get_tuning(P)["lane_chunk"] == lc
    _check(env, P, coef, pts)
    wl = W.unit_square_d1000(n_points=2000)
    P2 = F.fpe_precondition(wl.coeffs.re, wl.coeffs.im)
    F.fpe_set_tuning(P2, lw, lc)
    _check(env, P2, wl.coeffs, wl.points)


def test_autotune_single(env):
    torch, F = env
    rng = np.random.default_rng(32)
    coef = W.unit_disk_complex(1 << 16, rng)
    pts = W.sphere_points(1 << 15, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    zr = torch.from_numpy(pts.re).cuda()
    zi = torch.from_numpy(pts.im).cuda()
    best = F.fpe_autotune(P, zr, zi)
    assert best["long_window"] in GRID_LW and best["lane_chunk"] in GRID_LC and best["ms"] > 0.0
    assert F.fpe_get_tuning(P) == best
    lam = oracle.log2_abs(pts.re, pts.im)
    sample = np.concatenate([np.argsort(np.abs(lam))[:64], rng.choice(pts.n, 128, replace=False)])
    _check(env, P, coef, pts, sample)


def test_autotune_batch_and_graph(env):
    torch, F = env
    wls = W.batched_lognormal(n_poly=48, pts_per_poly=256, seed=33, dmax=1 << 14)
    offs = np.concatenate([[0], np.cumsum([w.points.n for w in wls])]).astype(np.int64)
    zre = np.concatenate([w.points.re for w in wls])
    zim = np.concatenate([w.points.im for w in wls])
    polys = [F.fpe_precondition(w.coeffs.re, w.coeffs.im) for w in wls]
    B = F.fpe_batch_create(polys, offs)
    zr = torch.from_numpy(zre).cuda()
    zi = torch.from_numpy(zim).cuda()
    best = F.fpe_batch_autotune(B, zr, zi)
    assert best["long_window"] in GRID_LW and best["lane_chunk"] in GRID_LC
    out = F.empty_out(B.n)
    F.fpe_batch_eval(B, zr, zi, out=out)
    torch.cuda.synchronize()
    ref = out.cpu().numpy().copy()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        F.fpe_batch_eval(B, zr, zi, out=out, stream=s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.int64), ref.view(np.int64))
    F.fpe_batch_sync(B)
    for i in (0, 7, 23, 47):
        w = wls[i]
        pre = oracle.precondition(w.coeffs, 53)
        vals, _ = oracle.fpe_eval(pre, w.points.re, w.points.im, with_S=True)
        Q, SQ = vals
        r = error_ratio(ref[offs[i]:offs[i + 1]], Q, SQ, TOL_FP64 * 31 / 32)
        assert r.max() <= 1.0, (i, r.max())
