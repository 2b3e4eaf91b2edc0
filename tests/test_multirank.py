"""Host logic of the multi-GPU (replicas / weak scaling) bench path on CPU:
two gloo ranks own disjoint wavepacket seeds and agree on the slowest rank's
time.  No data-path collective exists."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.shard_seeds(rank, 5)
    t = bench.max_over_ranks(10.0 + rank)
    out[rank] = (seeds, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time():
    world = 2
    port = 29500 + os.getpid() % 2000
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, t0 = res[0]
    s1, t1 = res[1]
    assert set(s0).isdisjoint(s1) and len(s0) == len(s1) == 5
    assert t0 == t1 == 11.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.shard_seeds(0, 3) == [0, 1, 2]
