"""Serving (continuous batching) on the GPU.

Requests of different collectives, vrank counts, dtypes and sizes are queued
at once; the server admits them as gangs and budget free up.  Every result
must equal the oracle for the plan the server reports, and requests re-run
alone must give the same bits as in the mix.  While a batching server runs its
kernel occupies the SMs, so inputs are prepared before it starts and outputs
are read back with copies only.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Server, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TYPESTR = {"fp32": "<f4", "bf16": "<i2", "fp16": "<f2", "int32": "<i4"}
NPDT = {"fp32": np.float32, "bf16": np.uint16, "fp16": np.float16, "int32": np.int32}


class _Dev:
    """A raw device pointer seen as a 1-D array (no copy)."""

    def __init__(self, ptr, n, dtype):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": TYPESTR[dtype],
                                         "data": (ptr, False), "version": 3}


def read_back(ptr, n, dtype):
    t = torch.as_tensor(_Dev(ptr, n, dtype), device="cuda")
    return t.cpu().numpy().view(NPDT[dtype]).copy()


def make_requests(seed, nreq, kmax, lo, hi):
    g = np.random.default_rng(seed)
    sizes = inputs.log_uniform_sizes(seed, nreq, lo, hi)
    reqs = []
    for i in range(nreq):
        coll = ("allreduce", "reducescatter", "allgather")[g.integers(3)]
        k = int(g.integers(2, kmax + 1))
        dtype = ("fp32", "bf16")[g.integers(2)]
        es = 4 if dtype == "fp32" else 2
        n = max(1, int(sizes[i]) // es)
        if coll != "allreduce":
            n = max(1, n // k)
        nin = k * n if coll == "reducescatter" else n
        xs = inputs.workload(seed * 7919 + i, k, nin, dtype, "normal")
        reqs.append(dict(coll=coll, k=k, dtype=dtype, n=n, xs=xs, op="sum"))
    return reqs


def run_server(reqs, **cfg):
    """Submit all requests at once, wait, return (outputs, plans, stats)."""
    sends = [[to_dev(x) for x in r["xs"]] for r in reqs]
    torch.cuda.synchronize()
    srv = Server(**cfg)
    try:
        tickets = [srv.submit(r["coll"], s, r["n"], r["dtype"], r["op"])
                   for r, s in zip(reqs, sends)]
        t0 = time.time()
        results = {}
        while len(results) < len(tickets):
            for r, t in zip(reqs, tickets):
                if t in results:
                    continue
                st, lat, plan, bufs = srv.query(t)
                if st in ("done", "failed"):
                    assert st == "done", (r["coll"], r["k"], st)
                    assert lat > 0
                    rn = r["k"] * r["n"] if r["coll"] == "allgather" else r["n"]
                    results[t] = ([read_back(bufs[q], rn, r["dtype"]) for q in range(r["k"])], plan)
                    srv.release(t)          # return the buffers to the budget at once
            assert time.time() - t0 < 120, "requests did not finish"
            time.sleep(0.001)
        outs = [results[t][0] for t in tickets]
        plans = [results[t][1] for t in tickets]
        stats = srv.stats()
    finally:
        srv.destroy()
    del sends
    return outs, plans, stats


def oracle_for(r, plan):
    dt, C = r["dtype"], plan["nchannels"]
    if r["coll"] == "allgather":
        return oracle.all_gather(r["xs"], C, chunk_for(plan["proto"], dt, SMALL_SLOTS, 1, True))
    ch = chunk_for(plan["proto"], dt, SMALL_SLOTS, 1)
    if r["coll"] == "allreduce":
        return oracle.all_reduce(r["xs"], dt, r["op"], C, ch)
    return oracle.reduce_scatter(r["xs"], dt, r["op"], C, ch)


CFG = dict(max_ranks=8, mem_budget=256 << 20, big_gang_channels=4, small_gangs=4,
           big_threshold=256 << 10, slot_bytes=SMALL_SLOTS, idle_timeout_sec=20.0)


@pytest.mark.parametrize("mode", ["batch", "streams"])
def test_serving_results_exact_and_same_alone(mode):
    reqs = make_requests(5, 48, 8, 1024, 2 << 20)
    outs, plans, stats = run_server(reqs, mode=mode, **CFG)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["maxInflightBytes"] <= CFG["mem_budget"]
    assert any(p["nchannels"] > 1 for p in plans)   # large requests spread over several channels
    for r, o, p in zip(reqs, outs, plans):
        want = oracle_for(r, p)
        for q in range(r["k"]):
            assert_same(o[q], want[q], f"{r['coll']} k={r['k']} n={r['n']} rank {q}")
    # the same requests alone, each on a fresh server, give the same bits
    for i in (0, 7, 19, 33):
        o1, p1, _ = run_server([reqs[i]], mode=mode, **CFG)
        assert p1[0] == plans[i]
        for q in range(reqs[i]["k"]):
            assert_same(o1[0][q], outs[i][q], f"request {i} alone vs in the mix, rank {q}")


@pytest.mark.parametrize("mode", ["batch", "streams"])
def test_serving_respects_memory_budget(mode):
    reqs = make_requests(9, 24, 8, 256 << 10, 1 << 20)
    budget = 24 << 20
    cfg = dict(CFG, mem_budget=budget)
    outs, plans, stats = run_server(reqs, mode=mode, **cfg)
    assert stats["completed"] == len(reqs)
    assert 0 < stats["maxInflightBytes"] <= budget


def test_plain_mode_exact():
    reqs = make_requests(11, 16, 8, 1024, 1 << 20)
    outs, plans, stats = run_server(reqs, mode="plain", **CFG)
    assert stats["completed"] == len(reqs)
    for r, o, p in zip(reqs, outs, plans):
        want = oracle_for(r, p)
        for q in range(r["k"]):
            assert_same(o[q], want[q], f"plain {r['coll']} k={r['k']} rank {q}")


def test_streams_and_plain_give_the_same_bits():
    """Plans depend on the request alone: the lanes of the streams mode and
    one launch per request produce identical results."""
    reqs = make_requests(13, 20, 8, 1024, 4 << 20)
    o1, p1, _ = run_server(reqs, mode="streams", **CFG)
    o2, p2, _ = run_server(reqs, mode="plain", **CFG)
    assert p1 == p2
    for i in range(len(reqs)):
        for q in range(reqs[i]["k"]):
            assert_same(o1[i][q], o2[i][q], f"request {i} rank {q}")
