"""The multi-GPU path of bench.py on CPU: two ranks over gloo combine their
figures as the driver expects (timed region: maximum over ranks; units:
sum over ranks); the shards cudisc_partition gives cover every cell once,
and cells integrated shard by shard (here by the FP64 oracle, one shard per
rank) equal one whole-grid integration bitwise, since cells evolve
independently during a coagulation call (no collective on the data path)."""
import os
import socket

import numpy as np
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


def _shard_rank(rank, world, port, scaling, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_2402_18471_b300 import synth
    if scaling == "strong":
        d = _small_disc()
        # costs as a calibration step measures them: accepted substeps per cell
        cost = O.Oracle(d).step(d.rho0, d.t_span)["n_acc"].astype(np.float64)
        b = bench.strong_bounds(d, world, cost)
        mine = np.arange(b[rank], b[rank + 1])
        part = d.subset(mine)
        y = O.Oracle(part).step(part.rho0, part.t_span)["rho"]
        item = (mine.tolist(), y)
    else:
        discs = bench.weak_shard("grid_128x64_N100", rank, world)
        assert len(discs) == 1
        dd = discs[0].subset(np.arange(0, 8192, 2048))
        dd.t_span = 30.0 * synth.CONST["yr"]
        y = O.Oracle(dd).step(dd.rho0, dd.t_span)["rho"]
        item = (discs[0].rho_gas[:64].tolist(), y)
    got = [None] * world
    dist.all_gather_object(got, item)
    if rank == 0:
        out["parts"] = got
    dist.barrier()
    dist.destroy_process_group()


def _small_disc():
    from paper_2402_18471_b300 import synth
    return synth.make_disc(5, 7, 14, 1e-5, 0.1, 5.0, 60.0, 30.0, seed=3, rho_pert=0.1)


def _spawn(scaling):
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, port, scaling, out), nprocs=world, join=True)
        return out["parts"]


def test_strong_shards_cover_cells_once_and_equal_the_whole_run(oracle_mod):
    parts = _spawn("strong")
    d = _small_disc()
    cells = np.concatenate([np.asarray(c, dtype=int) for c, _ in parts])
    assert np.array_equal(cells, np.arange(d.n_cells))          # each cell exactly once, in order
    assert all(len(c) > 0 for c, _ in parts)
    y = np.concatenate([np.asarray(r) for _, r in parts])
    whole = oracle_mod.Oracle(d).step(d.rho0, d.t_span)["rho"]
    assert np.array_equal(y, whole)                               # bitwise


def test_weak_shards_are_distinct_discs(oracle_mod):
    """Weak scaling: one disc of the workload per rank, each with its own
    seeded gas perturbations (rank 0 has the named workload itself)."""
    import bench
    parts = _spawn("weak")
    assert len(parts) == 2 and all(np.all(np.isfinite(np.asarray(r))) for _, r in parts)
    assert parts[0][0] != parts[1][0]
    assert parts[0][0] == bench.make_disc("grid_128x64_N100", 0).rho_gas[:64].tolist()
