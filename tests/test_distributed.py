"""Multi-process host logic on CPU (gloo, world size 2): model partition and
the throughput aggregation bench.py uses for N > 1 ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2304_11274_gb300 import synth
from paper_2304_11274_gb300.distributed import aggregate, partition


def test_partition_covers_every_model_once_and_balances():
    shapes = synth.ensemble_shapes()
    sizes = [a * b * c for a, b, c in shapes]
    for world in (1, 2, 3, 4, 8):
        parts = [partition(sizes, world, r) for r in range(world)]
        flat = sorted(m for p in parts for m in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[m] for m in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest model
        assert max(loads) - sum(loads) / world <= max(sizes)
    with pytest.raises(ValueError):
        partition(sizes, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shapes = synth.ensemble_shapes(count=10, nxy=(8, 20), nz=(4, 9))
        sizes = [a * b * c for a, b, c in shapes]
        mine = partition(sizes, world, rank)
        cells = sum(sizes[m] for m in mine)
        secs = 0.5 + rank  # a rank-dependent "time"
        total, worst = aggregate(cells, secs)
        out[rank] = (mine, cells, total, worst)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    sizes = [a * b * c for a, b, c in synth.ensemble_shapes(count=10, nxy=(8, 20), nz=(4, 9))]
    assert sorted(res[0][0] + res[1][0]) == list(range(10))
    assert res[0][2] == res[1][2] == sum(sizes)
    assert res[0][3] == res[1][3] == 1.5  # the max over ranks


# ---------------------------------------------------------------- z-slabs of one grid

def test_slab_bounds_cover_every_plane_once_with_halos():
    """Host logic of the slab decomposition (the C ABI's tpfa_slab_bounds):
    contiguous owned ranges covering [0, nz) once, sizes differing by at most
    one plane, halos one plane wide where a neighbouring slab exists."""
    from paper_2304_11274_gb300.api import slab_bounds
    from paper_2304_11274_gb300._capi import TPFAError
    for nz in (1, 2, 7, 11, 256):
        for parts in range(1, min(nz, 9) + 1):
            b = [slab_bounds(nz, parts, r) for r in range(parts)]
            assert b[0][0] == 0 and b[-1][1] == nz
            for (k0, k1, e0, e1), nxt in zip(b, b[1:] + [None]):
                assert k1 > k0
                if nxt is not None:
                    assert nxt[0] == k1
                assert e0 == max(k0 - 1, 0) and e1 == min(k1 + 1, nz)
            sizes = [k1 - k0 for k0, k1, _, _ in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(TPFAError):
        slab_bounds(4, 5, 0)  # more slabs than planes
    with pytest.raises(TPFAError):
        slab_bounds(4, 2, 2)


def _slab_worker(rank, world, port, nz, out):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2304_11274_gb300.api import slab_bounds
    from paper_2304_11274_gb300.distributed import slab_halo_exchange
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny = 5, 3
        nxy = nx * ny
        whole = torch.arange(nz * nxy, dtype=torch.float64) * 1.5 + 7.0  # plane k holds distinct values
        k0, k1, e0, e1 = slab_bounds(nz, world, rank)
        p = whole[e0 * nxy:e1 * nxy].clone()
        if k0 > e0:
            p[:nxy] = float("nan")  # the halo planes start unknown
        if e1 > k1:
            p[-nxy:] = float("nan")
        slab_halo_exchange(p, nxy, k0, k1, e0, e1, rank, world)
        out[rank] = bool(torch.equal(p, whole[e0 * nxy:e1 * nxy]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nz", [(2, 9), (3, 7)])
def test_slab_halo_exchange_with_gloo(world, nz):
    """Each rank's halo planes receive exactly the neighbouring slabs'
    boundary planes of the whole grid (point-to-point exchange, gloo)."""
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_slab_worker, args=(world, port, nz, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {r: True for r in range(world)}
