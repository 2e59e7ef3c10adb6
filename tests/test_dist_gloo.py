"""Multi-process host logic on CPU (gloo, world size 2): the benchmark's job time is the
maximum over ranks, and every replica solves its own set of densities.  Replicas run
independently; the maximum is the only cross-rank step of the benchmark."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = bench.max_over_ranks(values[rank], dist)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    world = 2
    values = [3.5, 1.25]
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, values, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == max(values) and out[1] == max(values)


def _slice_worker(rank, world, port, rhos, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.rank_densities(rhos, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out[rank] = gathered
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_solve_disjoint_density_sets_gloo():
    """Every rank builds its own batch: rank 0 the workload's densities, the others sets of the
    same shape that share no density with any other rank (the ranks agree on the layout)."""
    import torch.multiprocessing as mp
    import bench
    world = 2
    rhos = list(bench.WORKLOADS[bench.DEFAULT_WORKLOAD][1])
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_slice_worker, args=(world, port, rhos, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    sets = out[0]
    assert sets[0] == rhos
    assert all(len(x) == len(rhos) for x in sets)
    flat = [r for x in sets for r in x]
    assert len(set(flat)) == len(flat)


def test_rank_densities_disjoint_at_eight_ranks():
    import bench
    rhos = list(bench.WORKLOADS[bench.DEFAULT_WORKLOAD][1])
    flat = [r for k in range(8) for r in bench.rank_densities(rhos, k)]
    assert len(set(flat)) == len(flat) and all(r > 0 for r in flat)
