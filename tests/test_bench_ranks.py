"""The replicas-only multi-GPU path of bench.py on the CPU: two gloo ranks
(one replica each) combine into the whole-job figures, the sum of the
particle-steps and the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = [3.0e9, 5.0e9][rank]
    ms = [1200.0, 1500.0][rank]
    out[rank] = bench.aggregate_ranks(units, ms, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_units_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (8.0e9, 1500.0)


def test_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(7, 2.5, "cpu") == (7.0, 2.5)
