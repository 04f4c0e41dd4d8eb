"""Multi-rank logic of bench.py on CPU (gloo, world size 2): ranks get
disjoint seeded shards, the step time is the max over ranks, and the
whole-job rate counts the cells of every rank."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.workload(64, rank)
    fake_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mx = bench.reduce_max(fake_ms, dist, "cpu")
    out[rank] = (mx, int(b.q_codes[:32].sum()), b.cells())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 15.0          # max over ranks
    assert r0[1] != r1[1]                   # disjoint shards (different seeds)
    import bench
    v = bench.whole_job_gcups(r0[2], 2, 3, 15.0)
    assert np.isclose(v, r0[2] * 2 * 3 / 0.015 / 1e9)
    assert bench.shard_seed(0) != bench.shard_seed(1)
