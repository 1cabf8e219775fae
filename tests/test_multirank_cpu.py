"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with
its own seeded shard, timing reduced to the slowest rank."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2505_05940_gb300 import workloads as W
    ms = 100.0 + 25.0 * rank                      # the second rank is slower
    slowest = bench.max_over_ranks(ms, "cpu", world)
    _, inits = W.adjoint_plates(seed=bench.shard_seed(rank), n_inst=4, steps=16)
    d = [i.D for i in inits.instances]
    gathered = [None] * world
    dist.all_gather_object(gathered, d)
    value = bench.whole_job_value(world, 64, 200, 22050, slowest)
    out[rank] = (slowest, gathered, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_max():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        slowest, gathered, value = out[r]
        assert slowest == 125.0
        assert value == pytest.approx(2 * 64 * 200 * 22050 / 0.125)
        # each rank's shard is its own seeded draw: the two batches differ
        assert not np.allclose(gathered[0], gathered[1])
    assert out[0][1] == out[1][1]
