"""Replica bookkeeping for running the render path on several GPUs of one node.

The path shards without any exchange: views, frames and pixel tiles are independent and texel
sharing never leaves a warp. N processes (one per GPU) each render their own frames; the only
collectives are a barrier around the timed region and a max-reduction of the per-rank times.
"""
from __future__ import annotations


def frames_for_rank(rank: int, world: int, steps: int, base: int = 0) -> list[int]:
    """Frame indices rank `rank` renders in a `steps`-step timed region: disjoint across ranks,
    below 65536 (the frame field of the random stream)."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside world %d" % (rank, world))
    return [(base + rank * steps + i) % 65536 for i in range(steps)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over the default process group (the value itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
