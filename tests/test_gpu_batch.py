"""Batched launches (group calls) and the autotuner on the GPU.

Every call of a group must give, bit for bit, what the oracle gives for that
call with the plan the library reports for it; the batch must replay from a
CUDA graph; the tuner's table must drive Auto calls.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs
from paper_2507_04786_b300.binding import group

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NPT = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16, "int32": torch.int32}
DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}


def make_ops(seed, k, nops, lo_bytes, hi_bytes, colls=("allreduce", "reducescatter", "allgather",
                                                        "broadcast", "reduce")):
    """Random mixed group: collective, dtype, op, algo, protocol, size."""
    g = np.random.default_rng(seed)
    sizes = inputs.log_uniform_sizes(seed, nops, lo_bytes, hi_bytes)
    ops = []
    for i in range(nops):
        coll = colls[g.integers(len(colls))]
        dtype = ("fp32", "bf16", "int32", "fp16")[g.integers(4)]
        op = ("sum", "max")[g.integers(2)]
        proto = ("simple", "ll", "ll128", "auto")[g.integers(4)]
        algo = "tree" if coll == "allreduce" and g.integers(3) == 0 else "ring"
        es = 4 if dtype in ("fp32", "int32") else 2
        n = max(1, int(sizes[i]) // es - int(g.integers(0, 3)))   # ragged counts
        if coll in ("reducescatter", "allgather"):
            n = max(1, n // k)
        ops.append(dict(coll=coll, dtype=dtype, op=op, proto=proto, algo=algo, n=n,
                        root=int(g.integers(k)), seed=seed * 1000 + i))
    return ops


def issue(c, o, k):
    """Allocate and issue one call; returns (inputs, outputs) for checking."""
    dist, kw = DIST[o["dtype"]]
    n = o["n"]
    if o["coll"] == "reducescatter":
        xs = inputs.workload(o["seed"], k, k * n, o["dtype"], dist, **kw)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(n, dtype=NPT[o["dtype"]], device="cuda") for _ in range(k)]
        c.reduce_scatter(s, d, op=o["op"], algo="ring", proto=o["proto"])
    elif o["coll"] == "allgather":
        xs = inputs.workload(o["seed"], k, n, o["dtype"], dist, **kw)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(k * n, dtype=NPT[o["dtype"]], device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto=o["proto"])
    else:
        xs = inputs.workload(o["seed"], k, n, o["dtype"], dist, **kw)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(s[0]) for _ in range(k)]
        if o["coll"] == "allreduce":
            c.all_reduce(s, d, op=o["op"], algo=o["algo"], proto=o["proto"])
        elif o["coll"] == "broadcast":
            c.broadcast(s, d, root=o["root"], algo="ring", proto=o["proto"])
        else:
            d = [t if r == o["root"] else None for r, t in enumerate(d)]
            c.reduce(s, d, op=o["op"], root=o["root"], algo="ring", proto=o["proto"])
    return xs, s, d


def check(o, xs, d, plan, k):
    dt = o["dtype"]
    proto, C, cs = plan["proto"], plan["nchannels"], plan["chunkSteps"]
    if o["coll"] in ("allgather", "broadcast"):
        ch = chunk_for(proto, dt, SMALL_SLOTS, cs, byte_units=True)
        if o["coll"] == "allgather":
            want = oracle.all_gather(xs, C, ch)
        else:
            want = oracle.broadcast(xs, o["root"], C, ch)
        for r in range(k):
            assert_same(to_np(d[r], dt), want[r], f"{o} rank {r}")
        return
    ch = chunk_for(proto, dt, SMALL_SLOTS, cs)
    if o["coll"] == "allreduce":
        want = oracle.all_reduce(xs, dt, o["op"], C, ch, plan["algo"])
        for r in range(k):
            assert_same(to_np(d[r], dt), want[r], f"{o} plan {plan} rank {r}")
    elif o["coll"] == "reducescatter":
        want = oracle.reduce_scatter(xs, dt, o["op"], C, ch)
        for r in range(k):
            assert_same(to_np(d[r], dt), want[r], f"{o} plan {plan} rank {r}")
    else:
        want = oracle.reduce(xs, dt, o["op"], o["root"], C, ch)
        assert_same(to_np(d[o["root"]], dt), want, f"{o} plan {plan}")


@pytest.mark.parametrize("k,nch,nops", [(8, 8, 24), (4, 12, 40), (16, 4, 9), (3, 6, 64)])
def test_group_matches_oracle(k, nch, nops):
    c = Comm(k, nch, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    ops = make_ops(100 + k, k, nops, 256, 256 * 1024)
    issued = []
    with group():
        for o in ops:
            issued.append(issue(c, o, k))
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    plans = c.group_plans()
    assert len(plans) == nops
    for o, (xs, _, d), p in zip(ops, issued, plans):
        check(o, xs, d, p, k)
    c.destroy()


def test_group_replays_from_cuda_graph():
    """The batch launch captured in a CUDA graph replays with new inputs."""
    k, nch = 8, 8
    c = Comm(k, nch, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    c.prepare(algos=("ring", "tree"), protos=("simple", "ll", "ll128"))
    ops = make_ops(7, k, 16, 1024, 128 * 1024, colls=("allreduce", "reducescatter", "allgather"))
    issued = []
    with group():                       # one uncaptured run fixes the plans
        for o in ops:
            issued.append(issue(c, o, k))
    torch.cuda.synchronize()
    plans = c.group_plans()
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=stream):
        with group():
            for o, (xs, s, d) in zip(ops, issued):
                if o["coll"] == "allreduce":
                    c.all_reduce(s, d, op=o["op"], algo=o["algo"], proto=o["proto"])
                elif o["coll"] == "reducescatter":
                    c.reduce_scatter(s, d, op=o["op"], algo="ring", proto=o["proto"])
                else:
                    c.all_gather(s, d, algo="ring", proto=o["proto"])
    assert c.group_plans() == plans
    for rep in range(2):
        new = []
        for o, (xs, s, d) in zip(ops, issued):
            dist, kw = DIST[o["dtype"]]
            ys = inputs.workload(o["seed"] + 17 * (rep + 1), k, s[0].numel(), o["dtype"], dist, **kw)
            for t, y in zip(s, ys):
                t.copy_(to_dev(y))
            new.append(ys)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert c.async_error() == "vSuccess"
        for o, ys, (_, _, d), p in zip(ops, new, issued, plans):
            check(o, ys, d, p, k)
    c.destroy()


def test_tuner_table_drives_auto_calls():
    k, nch = 8, 8
    c = Comm(k, nch, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    c.tune(colls=("allreduce", "allgather"), max_bytes=1 << 20)
    tab = c.tune_table("allreduce")
    assert [e["bytes"] for e in tab] == [1024 * 4 ** i for i in range(6)]
    for e in tab:
        assert e["usec"] > 0 and 1 <= e["nchannels"] <= nch
        assert e["proto"] in ("simple", "ll", "ll128", "cluster", "direct") and e["algo"] in ("ring", "tree")
    assert len(c.tune_table("allgather")) == 6
    assert c.tune_table("reduce") == []
    # an Auto call takes the table's plan for its size bucket
    c.clear_plan()
    for e in tab:
        n = e["bytes"] // 4
        xs = inputs.workload(e["bytes"], k, n, "fp32", "normal")
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, algo="auto", proto="auto")
        torch.cuda.synchronize()
        p = c.last_plan()
        assert (p["algo"], p["proto"], p["nchannels"]) == (e["algo"], e["proto"], e["nchannels"])
        want = oracle.all_reduce(xs, "fp32", "sum", p["nchannels"],
                                 chunk_for(p["proto"], "fp32", SMALL_SLOTS, p["chunkSteps"]),
                                 p["algo"])
        for r in range(k):
            assert_same(to_np(d[r], "fp32"), want[r], f"bucket {e['bytes']} rank {r}")
    assert c.async_error() == "vSuccess"
    c.destroy()
