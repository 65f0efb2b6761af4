"""Multi-rank path of the bench on CPU (gloo, world size 2).

Each rank solves its own configurations (weak scaling): the instance sets
must be disjoint and the job time is the maximum over ranks; no collective
touches the data path.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import make_instance
    seeds = bench.rank_seeds(rank, 3)
    inst = make_instance("spheres8_grid7x14", seeds[0])
    t = bench.max_over_ranks(1.0 + rank)
    out[rank] = (seeds, t, float(inst.centers.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_bookkeeping():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    s0, t0, c0 = out[0]
    s1, t1, c1 = out[1]
    assert set(s0).isdisjoint(s1)
    assert t0 == t1 == 2.0
    assert c0 != c1                 # different configurations on the two ranks
