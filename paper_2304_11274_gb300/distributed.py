"""Host-side helpers for running the assembly on several GPUs (one process each).

The assembly has no exchange step between independent problems: an ensemble
is split across ranks model by model, and a single grid runs as one replica
per rank.  Only the timing reduction crosses ranks (a max of one scalar), so
nothing here is on the data path.
"""
from __future__ import annotations

import heapq


def partition(sizes, world: int, rank: int):
    """Indices of the models `rank` assembles: a greedy split of the models by
    cell count (largest first onto the least-loaded rank), deterministic for
    every rank, each model on exactly one rank.  Returns sorted indices."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(sizes)), key=lambda m: (-sizes[m], m))
    heap = [(0, r) for r in range(world)]
    owner = [0] * len(sizes)
    for m in order:
        load, r = heapq.heappop(heap)
        owner[m] = r
        heapq.heappush(heap, (load + sizes[m], r))
    return [m for m in range(len(sizes)) if owner[m] == rank]


def aggregate(local_cells: int, local_seconds: float, device=None):
    """(total cells over ranks, max seconds over ranks) through
    torch.distributed (any backend); a single process returns its own."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(local_cells), float(local_seconds)
    dev = device if device is not None else torch.device("cpu")
    cells = torch.tensor([float(local_cells)], dtype=torch.float64, device=dev)
    secs = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(cells, op=dist.ReduceOp.SUM)
    dist.all_reduce(secs, op=dist.ReduceOp.MAX)
    return int(cells.item()), float(secs.item())
