"""The multi-GPU path of bench.py on CPU: two ranks over gloo combine their
figures as the driver expects (timed region: maximum over ranks; units:
sum over ranks), and each rank's shard is the whole workload (weak scaling,
no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: its own timed region and units
    ms, e2e_s, sub, e2e_sub = bench.combine_ranks(dist, "cpu", 100.0 + 10 * rank, 2.0 + rank, 1000 + rank,
                                                  900 + 2 * rank)
    out[rank] = (ms, e2e_s, sub, e2e_sub)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_combine_over_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (110.0, 3.0, 2001, 1802)


def test_one_rank_passes_through():
    import bench
    assert bench.combine_ranks(None, "cpu", 5.0, 1.0, 7, 3) == (5.0, 1.0, 7, 3)
