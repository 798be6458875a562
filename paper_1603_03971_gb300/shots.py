"""Shots as the data-parallel unit: one process per GPU runs its own shots.

Shots are independent (each is a forward modelling plus a receiver
propagation with imaging), so ranks share nothing while they run. The one
exchange step of multi-shot RTM is the stack: the per-shot images are summed
into one image, here by a single all-reduce at the end.
"""
from __future__ import annotations

from typing import List, Tuple

import torch


def assign_shots(nshots: int, rank: int, world: int) -> List[int]:
    """Shots of one rank: a contiguous block, the first ``nshots % world``
    ranks taking one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(nshots, world)
    start = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return list(range(start, start + count))


def shot_source(shot: int, nshots: int, nx: int, ny: int, z: int) -> Tuple[int, int, int]:
    """Source position of shot ``shot`` of ``nshots`` on a line along x
    through the model centre, at depth index ``z``."""
    x = int(round((shot + 0.5) * nx / nshots))
    return (min(max(x, 0), nx - 1), ny // 2, z)


def stack_images(image: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the ranks' images in place (the multi-shot stack)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(image, op=dist.ReduceOp.SUM, group=group)
    return image


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """Largest value over all ranks (the job's wall time is its slowest rank)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
