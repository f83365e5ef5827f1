"""Views spread over ranks, one process per GPU.

Each view is an independent render of the shared Gaussians: the image of view v depends only on its pose and the
Gaussians (eqs. 3-8), and its adjoint only on that image's upstream gradient. A multi-GPU run therefore replicates
the scene on every rank and gives each rank its own contiguous slice of the batch of views; nothing crosses ranks on
the data path. Timing across ranks takes the slowest one.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def view_range(num_views: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of the views that `rank` renders out of `num_views`; the first num_views % world ranks get one
    extra view, so every view is rendered exactly once."""
    if world < 1 or not 0 <= rank < world or num_views < 0:
        raise ValueError(f"bad partition: {num_views} views, world {world}, rank {rank}")
    base, extra = divmod(num_views, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over the ranks of the default process group (the value itself without one)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
