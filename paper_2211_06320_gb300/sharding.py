"""Point sharding across ranks (one process per GPU).

Evaluation points are independent (§8.1: the algorithm is embarrassingly
parallel over points), so a multi-GPU run gives each rank a contiguous slice
of the points, evaluates it locally with no collective on the data path, and
at most gathers the results once at the end.  The polynomial itself is
replicated: every rank preconditions the same coefficients.
"""
from __future__ import annotations

from typing import Callable, Tuple


def shard_bounds(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's slice of n points; slices differ by at most one
    point and cover [0, n) in rank order."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def evaluate_sharded(evaluate: Callable, z_re, z_im, group=None):
    """Evaluate this rank's slice of the points with `evaluate(z_re, z_im) ->
    (m, 3) tensor` and all-gather the slices in rank order (one collective,
    after the evaluation).  Works on any torch.distributed backend; the
    tensors' device must suit it (CPU for gloo, CUDA for NCCL)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = int(z_re.shape[0])
    a, b = shard_bounds(n, rank, world)
    local = evaluate(z_re[a:b], None if z_im is None else z_im[a:b])
    sizes = [shard_bounds(n, r, world) for r in range(world)]
    width = max(s[1] - s[0] for s in sizes)
    pad = torch.zeros((width, local.shape[1]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][:sizes[r][1] - sizes[r][0]] for r in range(world)], dim=0)


def max_over_ranks(seconds: float, device="cpu", group=None) -> float:
    """The slowest rank's time: a weak-scaling step ends when every rank is done."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
