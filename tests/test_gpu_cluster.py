"""GPU parity of the cluster protocol (LL lines in distributed shared memory):
every collective through the C ABI against the CPU oracle, bit-exact.

To the oracle the cluster protocol is LL with 8 KiB slots (4 KiB of data per
FIFO step): the partition, the step tables and the fold order are the same.
Auto plans pick it on 2..16 vranks up to 256 KiB per rank.
Sizes span one to many FIFO steps, several chunks and ragged tails, on 2 to
16 vranks (16 is the largest cluster).
"""
import time

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, VcommError, group, inputs

from gpu_util import assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}
SIZES = [1, 5, 1023, 1025, 3 * 4096 + 7, 50003]

_comms = {}


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    assert torch.cuda.is_available()
    yield
    for c in _comms.values():
        c.destroy()
    _comms.clear()


def get_comm(k, C):
    if (k, C) not in _comms:
        _comms[(k, C)] = Comm(k, C, timeout_sec=10.0)
    return _comms[(k, C)]


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def chunk(dtype, steps, byte_units=False):
    return chunk_for("cluster", dtype, None, steps, byte_units=byte_units)


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max"),
                                      ("int32", "sum"), ("fp32", "max")])
@pytest.mark.parametrize("k,C,steps", [(2, 1, 1), (3, 2, 3), (5, 3, 2), (8, 2, 1), (16, 1, 3)])
def test_ring_allreduce(dtype, op, k, C, steps):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=steps)
    for n in SIZES:
        xs = data(n + k, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo="ring", proto="cluster")
        finish(c)
        assert c.last_plan()["proto"] == "cluster"
        want = oracle.all_reduce(xs, dtype, op, C, chunk(dtype, steps))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("int32", "max")])
@pytest.mark.parametrize("k,C,steps", [(2, 1, 1), (3, 1, 2), (4, 2, 1), (8, 2, 4), (11, 1, 1),
                                       (16, 2, 2)])
def test_tree_allreduce(dtype, op, k, C, steps):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=steps)
    for n in SIZES:
        xs = data(3 * n + k, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo="tree", proto="cluster")
        finish(c)
        p = c.last_plan()
        assert (p["algo"], p["proto"]) == ("tree", "cluster")
        want = oracle.all_reduce(xs, dtype, op, C, chunk(dtype, steps), "tree")
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("fp16", "sum"), ("int32", "max")])
@pytest.mark.parametrize("k,C", [(2, 1), (5, 2), (16, 3)])
def test_reduce_scatter(dtype, op, k, C):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    for m in (1, 777, 4099):
        xs = data(m + 11 * k, k, k * m, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.reduce_scatter(s, d, op=op, algo="ring", proto="cluster")
        finish(c)
        want = oracle.reduce_scatter(xs, dtype, op, C, chunk(dtype, 1))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"m={m} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
@pytest.mark.parametrize("k,C,steps", [(2, 1, 1), (6, 2, 3), (16, 2, 1)])
def test_all_gather(dtype, k, C, steps):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=steps)
    for m in (1, 999, 5000):
        xs = data(m + 5 * k, k, m, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(k * m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto="cluster")
        finish(c)
        want = oracle.all_gather(xs, C, chunk(dtype, steps, byte_units=True))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"m={m} rank {r}")
            assert_same(to_np(d[r], dtype), np.concatenate(xs), f"m={m} rank {r} vs concat")
    c.clear_plan()


@pytest.mark.parametrize("k,C,root", [(2, 1, 1), (5, 2, 0), (8, 1, 6), (16, 3, 9)])
def test_broadcast(k, C, root):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=2)
    for n in (1, 3000, 40001):
        xs = data(n + root, k, n, "fp16")
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.broadcast(s, d, root=root, algo="ring", proto="cluster")
        finish(c)
        for r in range(k):
            assert_same(to_np(d[r], "fp16"), xs[root], f"n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("int32", "max"), ("bf16", "sum")])
@pytest.mark.parametrize("k,C,root", [(2, 1, 0), (5, 2, 3), (16, 1, 15)])
def test_reduce(dtype, op, k, C, root):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=3)
    for n in (1, 2049, 30011):
        xs = data(n + 7 * root, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(s[0]) if r == root else None for r in range(k)]
        c.reduce(s, d, op=op, root=root, algo="ring", proto="cluster")
        finish(c)
        want = oracle.reduce(xs, dtype, op, root, C, chunk(dtype, 3))
        assert_same(to_np(d[root], dtype), want, f"n={n}")
    c.clear_plan()


def test_in_place_and_single_rank():
    # in-place AllReduce on 4 vranks; a single-rank communicator copies
    k, n = 4, 20000
    xs = data(5, k, n, "fp32")
    c = get_comm(k, 2)
    s = [to_dev(x) for x in xs]
    c.all_reduce(s, s, op="sum", algo="ring", proto="cluster")
    finish(c)
    p = c.last_plan()
    want = oracle.all_reduce(xs, "fp32", "sum", p["nchannels"], chunk("fp32", p["chunkSteps"]))
    for r in range(k):
        assert_same(to_np(s[r], "fp32"), want[r], f"rank {r}")
    c1 = get_comm(1, 2)
    x = to_dev(xs[0])
    y = torch.empty_like(x)
    c1.all_reduce([x], [y], proto="cluster")
    finish(c1)
    assert torch.equal(x, y)


def test_more_than_16_vranks_is_unsupported():
    c = get_comm(17, 1)
    s = [torch.ones(10, device="cuda") for _ in range(17)]
    d = [torch.empty_like(t) for t in s]
    with pytest.raises(VcommError) as e:
        c.all_reduce(s, d, proto="cluster")
    assert e.value.name == "vUnsupported"


def test_group_of_several_runs_as_ll():
    k, n = 4, 3000
    c = get_comm(k, 4)
    xs = [data(50 + i, k, n, "fp32") for i in range(3)]
    ss = [[to_dev(x) for x in x3] for x3 in xs]
    dd = [[torch.empty_like(t) for t in s] for s in ss]
    with group():
        for s, d in zip(ss, dd):
            c.all_reduce(s, d, op="sum", algo="ring", proto="cluster")
    finish(c)
    plans = c.group_plans()
    assert all(p["proto"] == "ll" for p in plans)
    for x3, d, p in zip(xs, dd, plans):
        want = oracle.all_reduce(x3, "fp32", "sum", p["nchannels"],
                                 chunk_for("ll", "fp32", None, p["chunkSteps"]))
        for r in range(k):
            assert_same(to_np(d[r], "fp32"), want[r], f"rank {r}")


@pytest.mark.parametrize("algo", ["ring", "tree"])
def test_lost_vrank_times_out(algo):
    """A vrank that never takes part: its peers' bounded waits run out, the
    host reads vTimeout, and the device stays usable."""
    k = 4
    c = Comm(k, 2, timeout_sec=0.2)
    s = [torch.ones(100000, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, algo=algo, proto="cluster")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    c.debug_skip_rank(1)
    t0 = time.time()
    c.all_reduce(s, d, algo=algo, proto="cluster")
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert c.async_error() == "vTimeout"
    c.destroy()
    c2 = Comm(k, 2)
    c2.all_reduce(s, d, algo=algo, proto="cluster")
    torch.cuda.synchronize()
    assert c2.async_error() == "vSuccess"
    assert float(d[3][-1]) == float(k)
    c2.destroy()
