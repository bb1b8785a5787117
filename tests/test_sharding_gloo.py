"""Multi-rank host logic on CPU: two gloo ranks shard the points, evaluate
their slices (with the CPU oracle standing in for the GPU), gather, and agree
with a single-process evaluation; the weak-scaling time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_06320_gb300.sharding import evaluate_sharded, max_over_ranks, shard_bounds


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
        out = evaluate_sharded(_oracle_eval(coef, pre), torch.from_numpy(pts.re), torch.from_numpy(pts.im))
        t = max_over_ranks(0.5 + rank)
        if rank == 0:
            q.put((out.numpy(), t))
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
    got, t = q.get(timeout=240)
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
    assert t == 1.5
