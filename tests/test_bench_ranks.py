"""The benchmark's multi-GPU arithmetic with two ranks on CPU (gloo): replicas
run independently, the whole-job value is the units all ranks processed over
the slowest rank's time, and every rank sees the same result.  (The path has
no data-path collective; only these reductions cross ranks.)"""

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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)            # rank 0: 1000 units, rank 1: 2000 units
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one (15 ms)
    value, ms_max = bench.replica_throughput(dist, "cpu", units, ms)
    mx = bench.over_ranks(dist, 3.0 + rank, "max", "cpu")
    sm = bench.over_ranks(dist, 3.0 + rank, "sum", "cpu")
    out[rank] = (value, ms_max, mx, sm)
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        value, ms_max, mx, sm = out[rank]
        assert ms_max == 15.0
        assert abs(value - 3000.0 / 0.015) < 1e-6
        assert mx == 4.0 and sm == 7.0


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(None, 2.5, "max", "cpu") == 2.5
    value, ms = bench.replica_throughput(None, "cpu", 500.0, 10.0)
    assert ms == 10.0 and abs(value - 50000.0) < 1e-9
