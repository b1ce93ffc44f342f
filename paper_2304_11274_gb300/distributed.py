"""Host-side helpers for running the assembly on several GPUs (one process each).

An ensemble is split across ranks model by model (no exchange: the models
are independent).  One grid is split into z-slabs (api.Slab): before each
assembly every rank sends its first and last owned planes of pressure to the
neighbouring ranks and receives their boundary planes into its halo planes,
point to point (NCCL on GPUs, gloo on CPU); in-plane links never cross a
slab boundary, so that one plane each way is the whole exchange.  The
timing reduction (a max of one scalar) also crosses ranks.
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


def slab_halo_exchange(p, nxy: int, k0: int, k1: int, e0: int, e1: int, rank: int, world: int, group=None):
    """Fill the halo planes of this rank's slab pressure from the neighbouring
    ranks.  p holds the planes [e0, e1) of the grid (flattened, nxy values
    per plane) of slab [k0, k1) (api.slab_bounds(nz, world, rank)); rank r
    owns slab r.  Sends the first owned plane down and the last owned plane
    up, receives the neighbours' into planes e0 (below) and e1 - 1 (above);
    returns after every transfer completed."""
    import torch.distributed as dist

    plane = lambda k: p[(k - e0) * nxy:(k - e0 + 1) * nxy]
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, plane(k0), rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, plane(k0 - 1), rank - 1, group))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, plane(k1 - 1), rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, plane(k1), rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
