"""Query-row sharding of the curvature over several GPUs (one process each).

Every point's neighbours range over all N points, so each rank holds a full
replica of X and computes kNN + curvature for a contiguous block of query rows
(mecuco_curvature_range); the only exchange is assembling the per-rank blocks
of kappa, an all-gather of equal-length (padded) slices.  Process groups are
torch.distributed ones (NCCL on GPUs; the host logic is exercised with gloo).
"""
from __future__ import annotations

import torch


def row_range(rank: int, world: int, n: int) -> tuple[int, int]:
    """Contiguous block [begin, end) of n rows for `rank` of `world`; the blocks
    tile [0, n) and their sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_rows(local: torch.Tensor, n: int, group=None) -> torch.Tensor:
    """Concatenate every rank's block (first dimension, in rank order) into the
    full n-row tensor on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    b, e = row_range(rank, world, n)
    if local.shape[0] != e - b:
        raise ValueError("local block does not match this rank's row range")
    width = -(-n // world)  # the largest block
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: e - b] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: row_range(r, world, n)[1] - row_range(r, world, n)[0]] for r in range(world)])


def curvature_sharded(ctx, X: torch.Tensor, k: int, group=None, **kw) -> torch.Tensor:
    """kappa of all N rows of X (a replica on every rank): this rank computes its
    row block with mecuco_curvature_range, then the blocks are all-gathered."""
    import torch.distributed as dist
    n = X.shape[0]
    b, e = row_range(dist.get_rank(group), dist.get_world_size(group), n)
    local = ctx.mecuco_curvature_range(X, k, b, e, **kw)
    return gather_rows(local, n, group)
