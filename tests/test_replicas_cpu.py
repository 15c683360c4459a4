"""Multi-GPU runs are independent replicas (the collectives never leave one
GPU); the only cross-rank step is the timing aggregation of bench.py.  Checked
here with two gloo ranks on the CPU: barrier, max over ranks, job value."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    bench.barrier(world)
    ms = [2.0, 3.5][rank]
    m = bench.reduce_max(world, ms)
    v = bench.job_value(world, 256 << 20, 8, m)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    import bench
    want = 2 * bench.busbw(256 << 20, 8, 3.5e-3)
    for rank, m, v in res:
        assert m == 3.5
        assert abs(v - want) < 1e-9
    assert abs(want - 2 * (256 << 20) / 3.5e-3 * 2 * 7 / 8 / 1e9) < 1e-9
