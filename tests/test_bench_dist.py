"""The multi-rank path of bench.py on the CPU (gloo, world size 2): ranks agree on the slowest
rank's time and the whole-job throughput counts every rank's replica."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._barrier_sync(world)
    mx = bench._max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
    out[rank] = (mx, bench.job_throughput(1000, 4, world, mx))
    dist.destroy_process_group()


def test_two_ranks_agree_on_max_and_throughput():
    import random
    port = 29500 + random.randint(0, 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # 2 replicas x 1000 px x 4 steps in 20 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 4 / 0.020 / 1e9)


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.job_throughput(67108864, 10, 1, 10.0) == pytest.approx(67.108864)
