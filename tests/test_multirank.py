"""The multi-GPU path's host logic, run as two gloo ranks on the CPU: the
scenario shards and the whole-job reduction of bench.py (sums over ranks,
the slowest rank's time)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2406_07048_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tot = np.array([100.0 * (rank + 1), rank + 3, 5.0 + 2 * rank, 1e9, 7.0, 8.0, 9.0, 10.0 * (rank + 1)])
        dist.barrier()
        red = bench.reduce_over_ranks(tot, dist, torch.device("cpu"))
        out[rank] = red.tolist()
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        red = np.array(out[r])
        assert red[0] == 300.0 and red[1] == 3 + 4          # sums
        assert red[2] == 7.0                                  # the slowest rank's time
        assert red[3] == 2e9 and red[7] == 30.0


def test_shards_are_disjoint_and_rank_independent():
    n = 3
    a = synth.config3(n_scen=n, first=bench.shard_first(0, n))
    b = synth.config3(n_scen=n, first=bench.shard_first(1, n))
    both = synth.config3(n_scen=2 * n, first=0)
    # rank 1's scenarios are scenarios n..2n-1 of one big batch, not rank 0's
    assert np.array_equal(b.horizon, both.horizon[n:]) and np.array_equal(a.horizon, both.horizon[:n])
    assert np.array_equal(b.obs_d, both.obs_d[int(both.obs_begin[n]):])
    assert not np.array_equal(a.obs_center[:4], b.obs_center[:4])
