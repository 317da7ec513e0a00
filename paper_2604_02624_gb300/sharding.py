"""Wavelength sharding of one design across processes (one GPU per process).

Every channel of the design is independent until the thickness gradient,
which all channels share: a rank takes a contiguous range of channels,
normalises its loss by the design's total channel count (``n_lambda_total``)
and the ranks sum their losses and gradients with one all-reduce.  No field
data crosses ranks.
"""
from __future__ import annotations

from typing import Tuple

import torch


def shard_range(n_lambda_total: int, rank: int, world: int) -> Tuple[int, int]:
    """Channels [lo, hi) of ``rank``: contiguous, sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(n_lambda_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_step(grad: torch.Tensor, loss: float, group=None) -> float:
    """Sum the ranks' gradient shards in place and return the summed loss."""
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return loss
    packed = torch.tensor([loss], dtype=torch.float64, device=grad.device)
    dist.all_reduce(grad, group=group)
    dist.all_reduce(packed, group=group)
    return float(packed.item())
