"""Point sharding across ranks (one process per GPU).

Evaluation points are independent (§8.1: the algorithm is embarrassingly
parallel over points), so a multi-GPU run splits one shared point set over
the ranks, each evaluates its share locally with no collective on the data
path, and the results are gathered at most once at the end.  The polynomial
is replicated: every rank preconditions the same coefficients.

A point's work is its window length, which depends on log2|z| (def. LRN):
points near |z| = 1 (or near minus a cover slope) have the longest windows.
Contiguous slices of an ordered point set would hand one rank all of them.
The default split therefore sorts the points by lambda = log2|z|, cuts the
sorted order into world * buckets_per_rank buckets of equal count, and deals
the buckets to the ranks round-robin: every rank gets points from every
part of the lambda range, and within a bucket the windows are alike (the
same bucketing the evaluation itself uses to keep a warp's windows alike).
The work concentrates in the few buckets near |z| = 1, so the buckets must
be fine: with 64 per rank the ranks' total window lengths agree within 1%
on an ordered point set (16 per rank left 25-30% between ranks).
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np


def shard_bounds(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's contiguous slice of n points; slices differ by
    at most one point and cover [0, n) in rank order."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def lambda_of(z_re, z_im=None) -> np.ndarray:
    """log2|z| on the host (-inf at z = 0; non-finite points sort last)."""
    zr = np.asarray(z_re, dtype=np.float64)
    a = np.abs(zr) if z_im is None else np.hypot(zr, np.asarray(z_im, dtype=np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = np.log2(a)
    return np.where(np.isnan(lam), np.inf, lam)


def lambda_round_robin(z_re, z_im, rank: int, world: int, buckets_per_rank: int = 64) -> np.ndarray:
    """Indices (increasing) of rank's points: the points sorted by log2|z|
    (stable), cut into world * buckets_per_rank buckets of equal count,
    bucket b dealt to rank b mod world.  Every rank computes the same split."""
    if world < 1 or not (0 <= rank < world) or buckets_per_rank < 1:
        raise ValueError("bad shard arguments")
    n = int(np.asarray(z_re).shape[0])
    order = np.argsort(lambda_of(z_re, z_im), kind="stable")
    nb = world * buckets_per_rank
    edges = [shard_bounds(n, b, nb) for b in range(nb)]
    mine = [order[a:c] for b, (a, c) in enumerate(edges) if b % world == rank]
    idx = np.concatenate(mine) if mine else np.zeros(0, dtype=np.int64)
    return np.sort(idx)


def evaluate_sharded(evaluate: Callable, z_re, z_im, group=None, split: str = "lambda",
                     buckets_per_rank: int = 64):
    """Evaluate this rank's share of the points with `evaluate(z_re, z_im) ->
    (m, 3) tensor`, all-gather the shares (one collective, after the
    evaluation) and return the (n, 3) results in the caller's point order.
    split: "lambda" (lambda-sorted round-robin buckets, the default) or
    "contiguous".  Works on any torch.distributed backend; the tensors'
    device must suit it (CPU for gloo, CUDA for NCCL)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = int(z_re.shape[0])
    if split == "lambda":
        zr_h = z_re.detach().cpu().numpy()
        zi_h = None if z_im is None else z_im.detach().cpu().numpy()
        shares = [lambda_round_robin(zr_h, zi_h, r, world, buckets_per_rank) for r in range(world)]
    elif split == "contiguous":
        shares = [np.arange(*shard_bounds(n, r, world)) for r in range(world)]
    else:
        raise ValueError("split must be 'lambda' or 'contiguous'")
    idx = torch.from_numpy(shares[rank]).to(z_re.device)
    local = evaluate(z_re[idx], None if z_im is None else z_im[idx])
    width = max(len(s) for s in shares)
    pad = torch.zeros((width, local.shape[1]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = torch.empty((n, local.shape[1]), dtype=local.dtype, device=local.device)
    for r in range(world):
        out[torch.from_numpy(shares[r]).to(local.device)] = parts[r][:len(shares[r])]
    return out


def max_over_ranks(seconds: float, device="cpu", group=None) -> float:
    """The slowest rank's time: a step ends when every rank is done."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
