"""Host-side helpers for runs with one process per GPU (torch.distributed).

The product needs no exchange between GPUs: independent products (or independent problems of a
batch) are simply divided among the ranks.  What the ranks share is bookkeeping: a timed region
counts as long as its slowest rank, and a list of units is split into contiguous blocks."""
from __future__ import annotations

import torch


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The maximum of x over all ranks (x itself without an initialised process group).
    device: where the reduction runs ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_range(n: int, rank: int, world: int) -> range:
    """Rank's contiguous block of the units [0, n): block sizes differ by at most one, and the
    blocks follow the rank order."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))
