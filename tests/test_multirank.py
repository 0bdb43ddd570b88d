"""The replica path of bench.py on several ranks (world size 2, gloo on
CPU): the job's time is the slowest rank's and its iterations are summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 12.5][rank]
    iters = [5, 7][rank]
    t, n = bench.reduce_over_ranks(ms, iters, "cpu")
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (12.5, 12.0) and out[1] == (12.5, 12.0)


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(3.0, 4, "cpu") == (3.0, 4.0)
