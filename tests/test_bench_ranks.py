"""The multi-rank logic of bench.py on CPU: two gloo ranks, each with its own
problem, report the slowest rank's time and the whole job's throughput."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        rec = bench.rank_recipe("matern2d", 1000, rank)
        import synthdata
        x = synthdata.points_np(rec)
        out[rank] = (ms_max, bench.job_throughput(rec.n, world, ms_max), rec.seed, float(x[:10].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_independent_problems():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 15.0                         # max over ranks
    assert r0[1] == r1[1] == pytest.approx(2 * 1000 / 0.015)   # whole-job points/s
    assert r0[2] != r1[2] and r0[3] != r1[3]              # different seeds, different points
