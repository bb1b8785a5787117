"""Multi-rank host logic on CPU: two gloo ranks split one shared point set
(lambda-sorted round-robin buckets, and contiguous slices), evaluate their
shares (with the CPU oracle standing in for the GPU), gather, and agree with
a single-process evaluation; the step time is the slowest rank's.  The
lambda split balances the work (the window lengths) where contiguous slices
of an ordered point set do not."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_06320_gb300.sharding import (evaluate_sharded, lambda_of, lambda_round_robin, max_over_ranks,
                                             shard_bounds)


def test_shard_bounds_partition():
    for n in (0, 1, 5, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def test_lambda_round_robin_partition_and_balance():
    """The shares partition the points; every rank's share spans the whole
    lambda range; on points sorted by |z| the per-rank window work (the
    oracle's window lengths) is within 5% across ranks, where contiguous
    slices (three ranks or more) put the long windows near |z| = 1 on one."""
    import oracle
    import workloads as W
    rng = np.random.default_rng(3)
    coef = W.unit_square_complex(2000, rng)
    pts = W.sphere_points(20000, rng)
    order = np.argsort(np.hypot(pts.re, pts.im))  # an ordered point set
    zr, zi = pts.re[order], pts.im[order]
    pre = oracle.precondition(coef, 53)
    _, _, lo, hi = oracle.windows(pre.hk, pre.hs, pre.T, oracle.log2_abs(zr, zi))
    work = (hi - lo + 1).astype(np.float64)
    lam = lambda_of(zr, zi)
    for world in (2, 3, 8):
        shares = [lambda_round_robin(zr, zi, r, world) for r in range(world)]
        allidx = np.concatenate(shares)
        assert np.array_equal(np.sort(allidx), np.arange(zr.size))
        for s in shares:
            assert np.all(np.diff(s) > 0)
            assert lam[s].min() <= np.quantile(lam, 0.1) and lam[s].max() >= np.quantile(lam, 0.9)
        w = np.array([work[s].sum() for s in shares])
        assert w.max() / w.min() < 1.05, (world, w)
        wc = np.array([work[a:b].sum() for a, b in (shard_bounds(zr.size, r, world) for r in range(world))])
        if world >= 3:  # the middle slice holds |z| near 1: the imbalance the lambda split removes
            assert wc.max() / wc.min() > 1.5, (world, wc)
    with pytest.raises(ValueError):
        lambda_round_robin(zr, zi, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_eval(coef, pre):
    import oracle

    def ev(zr, zi):
        vals, _ = oracle.fpe_eval(pre, zr.numpy(), zi.numpy())
        # (re, im, e) rows like the library's fpe_xc64 (hi parts only)
        e = vals.e.astype(np.float64)
        return torch.from_numpy(np.stack([vals.re_hi, vals.im_hi, e], axis=1))
    return ev


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import workloads as W
        rng = np.random.default_rng(0)
        coef = W.unit_square_complex(300, rng)
        pts = W.sphere_points(1001, rng)
        pre = oracle.precondition(coef, 53)
        zr, zi = torch.from_numpy(pts.re), torch.from_numpy(pts.im)
        out = evaluate_sharded(_oracle_eval(coef, pre), zr, zi)
        out_c = evaluate_sharded(_oracle_eval(coef, pre), zr, zi, split="contiguous")
        t = max_over_ranks(0.5 + rank)
        if rank == 0:
            q.put((out.numpy(), out_c.numpy(), t))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharded_evaluation():
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, got_c, t = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(0)
    coef = W.unit_square_complex(300, rng)
    pts = W.sphere_points(1001, rng)
    pre = oracle.precondition(coef, 53)
    want = _oracle_eval(coef, pre)(torch.from_numpy(pts.re), torch.from_numpy(pts.im)).numpy()
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    assert np.array_equal(got_c, want)
    assert t == 1.5
