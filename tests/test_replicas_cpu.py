"""The N>1 path of bench.py is replicas only (independent copies of the workload, no data-path
collective): the timing is the maximum over ranks and the value is world * units / that time.
Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [1.25, 3.5][rank]                       # rank 1 is the slow one
    tmax = bench.world_max(t, dist, "cpu")
    value = bench.whole_job_value(1e6 * 10, world, tmax)
    dist.barrier()
    out[rank] = (tmax, value)
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    world = 2
    port = free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    tmax, value = out[0]
    assert tmax == 3.5
    assert value == pytest.approx(2 * 10 / 3.5)
