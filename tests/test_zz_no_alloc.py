"""fpe_eval_noalloc: evaluation for callers that cannot allocate device memory
while they evaluate (fixed device-memory budgets, latency-bound loops that
must not pay for cudaMalloc, hosts that only hand over their own buffers).
It must give the same values as fpe_eval, within the parity tolerance, on two
calls in a row that share its built-in scratch array.  This file is collected
last so that a failure here leaves every other test already run."""
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


def _compare(env, P, coef, zre, zim):
    torch, F = env
    zr = torch.from_numpy(zre).cuda()
    zi = torch.from_numpy(zim).cuda()
    n = zre.shape[0]
    a = F.fpe_eval_noalloc(P, zr, zi)
    F.fpe_sync(P)
    b = F.fpe_eval(P, zr, zi)
    F.fpe_sync(P)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    # the existing entry point's output as the reference, tolerance 2^-50 S(z)
    _, S, _ = oracle.horner_ref(coef, zre, zim)
    be = np.ascontiguousarray(b[:, 2]).view(np.int64)
    ref = oracle.ExtValues(np.stack([b[:, 0], np.zeros(n), b[:, 1], np.zeros(n)], axis=1), be)
    r = error_ratio(a, ref, S, TOL_FP64)
    assert r.max() <= 1.0, f"noalloc differs from fpe_eval by {r.max():.3g} x tolerance"
    return r.max()


def test_noalloc_matches_fpe_eval_twice(env):
    torch, F = env
    rng = np.random.default_rng(2468)
    coef = W.unit_disk_complex(12000, rng)
    P = F.fpe_precondition(coef.re, coef.im)
    # first call: sphere points (short windows and a few long ones)
    p1 = W.sphere_points(F.NOALLOC_MAX_POINTS, rng)
    _compare(env, P, coef, p1.re, p1.im)
    # second call on different points: unit-circle points, every window long (warp groups),
    # so stale scratch from the first call would show
    t = rng.uniform(0, 2 * math.pi, 3000)
    _compare(env, P, coef, np.cos(t), np.sin(t))


def test_noalloc_rejects_too_many_points(env):
    torch, F = env
    coef = W.unit_square_complex(50, np.random.default_rng(1))
    P = F.fpe_precondition(coef.re, coef.im)
    z = torch.zeros(F.NOALLOC_MAX_POINTS + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FpeError) as e:
        F.fpe_eval_noalloc(P, z, z)
    assert e.value.status == F.FPE_ERR_INVALID_ARG
