"""The multi-GPU benchmark path on CPU with two gloo ranks: every rank builds its own batch of the same size
(weak scaling, independent seeds), and the only collective is the MAX of the per-rank step times."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scs, _ = bench.workload("batch8", bench.rank_seed(4, 0), rank)
    sizes = [sc.n_verts for sc in scs]
    t = bench.max_over_ranks(1.0 + rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, (len(scs), sum(sizes), [sc.name for sc in scs]))
    out[rank] = (t, gathered)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    t0, g0 = out[0]
    t1, g1 = out[1]
    assert t0 == t1 == 2.0                       # MAX over ranks
    assert g0 == g1
    (n0, v0, names0), (n1, v1, names1) = g0
    assert n0 == n1 == 8                         # same batch size per rank (weak scaling)
    assert names0 != names1                      # independent instances
