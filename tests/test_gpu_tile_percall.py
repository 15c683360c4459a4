"""Single direct-protocol calls that the host hands to the tile engine (one
call as a one-op launch of kBatchTiles: AllReduce on 12..16 vranks,
ReduceScatter blocks that are not whole 16-byte units on up to 8 vranks),
with the size threshold lowered (VCOMM_TILE_MIN_BYTES) so
that oracle-sized inputs span many tiles: every element equal to the
oracle's for the reported plan and to the per-call kernels' bits (the
threshold raised out of reach); the launch list shows which kernel ran; a
captured graph of such a call replays with new inputs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def make_comm(k, C, tile_min):
    old = os.environ.get("VCOMM_TILE_MIN_BYTES")
    os.environ["VCOMM_TILE_MIN_BYTES"] = str(tile_min)
    try:
        return Comm(k, C, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    finally:
        if old is None:
            del os.environ["VCOMM_TILE_MIN_BYTES"]
        else:
            os.environ["VCOMM_TILE_MIN_BYTES"] = old


def run(c, coll, xs, n, dtype, op):
    s = [to_dev(x) for x in xs]
    d = [torch.full((n,), 7, dtype=s[0].dtype, device="cuda") for _ in xs]
    if coll == "allreduce":
        c.all_reduce(s, d, op=op, algo="ring", proto="direct")
    else:
        c.reduce_scatter(s, d, op=op, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    return [to_np(t, dtype) for t in d], c.last_plan()


def want(coll, xs, dtype, op, p):
    ch = chunk_for("direct", dtype, SMALL_SLOTS, p["chunkSteps"])
    if coll == "allreduce":
        return oracle.all_reduce(xs, dtype, op, p["nchannels"], ch)
    return oracle.reduce_scatter(xs, dtype, op, p["nchannels"], ch)


CASES = [("allreduce", 12, 200003, "fp32", "sum"), ("allreduce", 16, 300001, "bf16", "sum"),
         ("allreduce", 16, 65536, "int32", "max"), ("allreduce", 13, 100000, "fp16", "max"),
         # blocks that are not whole 16-byte units
         ("reducescatter", 3, 50001, "fp32", "sum"), ("reducescatter", 7, 30003, "bf16", "sum"),
         ("reducescatter", 8, 9999, "fp16", "max"), ("reducescatter", 4, 12345, "int32", "max"),
         # not routed (the per-call kernels on both sides)
         ("reducescatter", 8, 32768, "bf16", "max"), ("reducescatter", 16, 9999, "fp16", "max")]


@pytest.mark.parametrize("coll,k,n,dtype,op", CASES)
def test_routed_calls_exact_and_equal_to_per_call_kernels(coll, k, n, dtype, op):
    xs = data(1000 + k + n, k, k * n if coll == "reducescatter" else n, dtype)
    c1 = make_comm(k, 4, 16)
    got, p1 = run(c1, coll, xs, n, dtype, op)
    c2 = make_comm(k, 4, 1 << 62)
    ref, p2 = run(c2, coll, xs, n, dtype, op)
    assert p1 == p2
    w = want(coll, xs, dtype, op, p1)
    for r in range(k):
        assert_same(got[r], w[r], f"{coll} k={k} n={n} {dtype} {op} rank {r}")
        assert_same(got[r], ref[r], f"{coll} vs per-call kernels rank {r}")
    c1.destroy()
    c2.destroy()


def kernels(c, k, n):
    prof = pytest.importorskip("torch.profiler")
    s = [torch.ones(n, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    torch.cuda.synchronize()
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        c.all_reduce(s, d, algo="ring", proto="direct")
        torch.cuda.synchronize()
    assert c.async_error() == "vSuccess" and float(d[k - 1][-1]) == float(k)
    return [e.name for e in p.events()]


def test_launch_list_shows_the_route():
    c16 = make_comm(16, 4, 16)
    k16 = kernels(c16, 16, 100000)
    c16.destroy()
    if not k16:
        pytest.skip("the profiler recorded no CUDA kernels")
    assert any("kBatchTiles" in x for x in k16)
    c8 = make_comm(8, 4, 16)               # AllReduce on 8 vranks keeps the per-call kernels
    k8 = kernels(c8, 8, 100000)
    c8.destroy()
    assert not any("kBatchTiles" in x for x in k8)
    cbig = make_comm(16, 4, 1 << 62)       # below the threshold: the per-call kernels
    kbig = kernels(cbig, 16, 100000)
    cbig.destroy()
    assert not any("kBatchTiles" in x for x in kbig)


def test_routed_call_replays_from_a_graph():
    k, n = 16, 200000
    c = make_comm(k, 4, 16)
    xs1, xs2 = data(5, k, n, "fp32"), data(6, k, n, "fp32")
    s = [to_dev(x) for x in xs1]
    d = [torch.empty_like(t) for t in s]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c.all_reduce(s, d, algo="ring", proto="direct", stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        c.all_reduce(s, d, algo="ring", proto="direct", stream=stream)
    p = c.last_plan()
    for t, x in zip(s, xs2):
        t.copy_(torch.from_numpy(x))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    w = oracle.all_reduce(xs2, "fp32", "sum", p["nchannels"], chunk_for("direct", "fp32", SMALL_SLOTS,
                                                                        p["chunkSteps"]))
    for r in range(k):
        assert_same(to_np(d[r], "fp32"), w[r], f"graph replay rank {r}")
    c.destroy()
