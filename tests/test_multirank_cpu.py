"""The N>1 timing path of bench.py on CPU: two gloo ranks, MAX over ranks, whole-job value."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its timed region took (r + 1) * 100 ms for 3 steps of 1e9 pairs
    value, total = bench.aggregate((rank + 1) * 100.0, 10**9, 3, world, device="cpu")
    out[rank] = (value, total)
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_rank_aggregate_uses_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        value, total = out[r]
        assert total == pytest.approx(200.0)
        # 2 ranks x 3 steps x 1e9 pairs over 0.2 s = 30 Gpairs/s
        assert value == pytest.approx(30.0)
