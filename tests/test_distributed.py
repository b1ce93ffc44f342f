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
