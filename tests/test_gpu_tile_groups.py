"""Group calls of direct-protocol collectives as ONE launch of the tile engine
(kBatchTiles): every call's tiles laid end to end, CTA j taking tiles j,
j + grid, ...; tiles of 16-byte aligned buffers (and ReduceScatter blocks that
are not whole 16-byte units, through shifted windows) move by bulk copies
through shared memory, the rest take the register kernels' paths.

Each result must equal the oracle's for its reported plan and the bits of the
same group launched the older way (one register kernel per (dtype, op) class,
VCOMM_TILE_GROUPS=0); the launch list must show one kernel for the group; a
captured CUDA graph of the group replays with new inputs; groups the tile
engine does not take (more than 16 vranks, avg) still run.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, group, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def make_comm(k, C, tile_groups=True):
    old = os.environ.get("VCOMM_TILE_GROUPS")
    os.environ["VCOMM_TILE_GROUPS"] = "1" if tile_groups else "0"
    try:
        return Comm(k, C, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    finally:
        if old is None:
            del os.environ["VCOMM_TILE_GROUPS"]
        else:
            os.environ["VCOMM_TILE_GROUPS"] = old


def build_calls(k, seed, ncalls, sizes):
    rng = np.random.default_rng(seed)
    colls = ("allreduce", "reducescatter", "allgather", "broadcast", "reduce")
    calls = []
    for i in range(ncalls):
        coll = colls[i % 5]
        dtype = ("fp32", "bf16", "fp16", "int32")[int(rng.integers(4))]
        op = ("sum", "max")[int(rng.integers(2))]
        n = int(rng.choice(sizes))
        root = int(rng.integers(k))
        m = k * n if coll == "reducescatter" else n
        calls.append(dict(coll=coll, dtype=dtype, op=op, n=n, root=root, xs=data(seed * 100 + i, k, m, dtype)))
    return calls


def run_group(c, calls, k, off=0):
    outs = []
    with group():
        for cl in calls:
            s = [to_dev(x) for x in cl["xs"]]
            outn = cl["n"] if cl["coll"] != "allgather" else k * cl["n"]
            d = [torch.full((outn + off,), 3, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
            if cl["coll"] == "allreduce":
                c.all_reduce(s, d, op=cl["op"], algo="ring", proto="direct")
            elif cl["coll"] == "reducescatter":
                c.reduce_scatter(s, d, op=cl["op"], algo="ring", proto="direct")
            elif cl["coll"] == "allgather":
                c.all_gather(s, d, algo="ring", proto="direct")
            elif cl["coll"] == "broadcast":
                c.broadcast(s, d, root=cl["root"], algo="ring", proto="direct")
            else:
                d = [t if r == cl["root"] else None for r, t in enumerate(d)]
                c.reduce(s, d, op=cl["op"], root=cl["root"], algo="ring", proto="direct")
            outs.append((s, d))
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    return outs, c.group_plans()


def expected(cl, p, k):
    C, ch = p["nchannels"], chunk_for("direct", cl["dtype"], SMALL_SLOTS, p["chunkSteps"])
    xs = cl["xs"]
    if cl["coll"] == "allreduce":
        return oracle.all_reduce(xs, cl["dtype"], cl["op"], C, ch)
    if cl["coll"] == "reducescatter":
        return oracle.reduce_scatter(xs, cl["dtype"], cl["op"], C, ch)
    if cl["coll"] == "allgather":
        return [np.concatenate(xs)] * k
    if cl["coll"] == "broadcast":
        return [xs[cl["root"]]] * k
    w = [None] * k
    w[cl["root"]] = oracle.reduce(xs, cl["dtype"], cl["op"], cl["root"], C, ch)
    return w


@pytest.mark.parametrize("k,off", [(2, 0), (5, 0), (8, 0), (8, 1), (16, 0)])
def test_group_exact_and_equal_to_class_launches(k, off):
    calls = build_calls(k, 31 + k, 30, [1, 3, 17, 1000, 4099, 65537, 300001])
    c1 = make_comm(k, 4, tile_groups=True)
    o1, p1 = run_group(c1, calls, k, off)
    c2 = make_comm(k, 4, tile_groups=False)
    o2, p2 = run_group(c2, calls, k, off)
    assert p1 == p2 and len(p1) == len(calls)
    for cl, (s, d1), (_, d2), p in zip(calls, o1, o2, p1):
        want = expected(cl, p, k)
        for r in range(k):
            if want[r] is None:
                continue
            assert_same(to_np(d1[r], cl["dtype"]), want[r], f"{cl['coll']} {cl['dtype']} n={cl['n']} rank {r}")
            assert_same(to_np(d1[r], cl["dtype"]), to_np(d2[r], cl["dtype"]), f"{cl['coll']} vs class launches")
    c1.destroy()
    c2.destroy()


def test_group_is_one_launch():
    prof = pytest.importorskip("torch.profiler")
    k = 8
    calls = build_calls(k, 7, 20, [1000, 4099, 300001])
    c = make_comm(k, 4)
    run_group(c, calls, k)          # the group once, outside the profiler
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        run_group(c, calls, k)
        torch.cuda.synchronize()
    names = [e.name for e in p.events() if "kBatchTiles" in e.name or "kDirect" in e.name]
    if not names:
        pytest.skip("the profiler recorded no CUDA kernels")
    assert sum("kBatchTiles" in x for x in names) == 1 and not any("kDirect" in x for x in names), names
    c.destroy()


def test_group_replays_from_a_cuda_graph():
    k = 8
    c = make_comm(k, 4)
    sizes = [4099, 65537, 1 << 20]
    xs1 = [data(900 + i, k, n, "fp32") for i, n in enumerate(sizes)]
    xs2 = [data(950 + i, k, n, "fp32") for i, n in enumerate(sizes)]
    s = [[to_dev(x) for x in xs] for xs in xs1]
    d = [[torch.empty_like(t) for t in si] for si in s]
    stream = torch.cuda.Stream()

    def grp():
        with group():
            for si, di in zip(s, d):
                c.all_reduce(si, di, op="sum", algo="ring", proto="direct", stream=stream)

    with torch.cuda.stream(stream):
        grp()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        grp()
    plans = c.group_plans()
    for si, xs in zip(s, xs2):        # new inputs, same buffers
        for t, x in zip(si, xs):
            t.copy_(torch.from_numpy(x))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    for di, xs, p in zip(d, xs2, plans):
        want = oracle.all_reduce(xs, "fp32", "sum", p["nchannels"], chunk_for("direct", "fp32", SMALL_SLOTS,
                                                                              p["chunkSteps"]))
        for r in range(k):
            assert_same(to_np(di[r], "fp32"), want[r], f"graph replay rank {r}")
    c.destroy()


def test_groups_the_tile_engine_does_not_take():
    """More than 16 vranks, or avg: the group runs on the per-class kernels."""
    for k, op in ((20, "sum"), (4, "avg")):
        calls = [dict(coll="allreduce", dtype="fp32", op=op, n=4099, root=0, xs=data(77 + k, k, 4099, "fp32"))]
        c = make_comm(k, 2)
        o, p = run_group(c, calls, k)
        want = oracle.all_reduce(calls[0]["xs"], "fp32", op, p[0]["nchannels"],
                                 chunk_for("direct", "fp32", SMALL_SLOTS, p[0]["chunkSteps"]))
        for r in range(k):
            assert_same(to_np(o[0][1][r], "fp32"), want[r], f"k={k} {op} rank {r}")
        c.destroy()
