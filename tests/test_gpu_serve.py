"""Serving (continuous batching) on the GPU, for every protocol.

Requests of different collectives, vrank counts (2..16), dtypes and sizes are
queued at once; the server admits them as gangs, lanes and budget free up.
Every result must equal the oracle for the plan the server reports, and
requests re-run alone must give the same bits as in the mix.  Each test runs
with the paper's FIFO protocols (Simple, LL, LL128: the resident gangs'
flag-polled path) and with Auto (the direct protocol), in the three modes
(resident gangs, lanes of streams, one launch per request).  While a batching
server runs its kernel occupies the SMs, so inputs are prepared before it
starts and outputs are read back with copies only.
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
PROTOS = ["simple", "ll", "ll128", "auto"]
MODES = ["batch", "streams", "plain"]
# continuous-batching modes and protocols: resident gangs and lanes of streams
# run every protocol; the tile kernel runs the direct protocol (Auto) only
BATCHING = [(m, p) for m in ("batch", "streams") for p in PROTOS] + [("tiles", "auto")]


class _Dev:
    """A raw device pointer seen as a 1-D array (no copy)."""

    def __init__(self, ptr, n, dtype):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": TYPESTR[dtype],
                                         "data": (ptr, False), "version": 3}


def read_back(ptr, n, dtype, idx=None):
    t = torch.as_tensor(_Dev(ptr, n, dtype), device="cuda")
    if idx is not None:
        t = t[torch.from_numpy(idx).cuda()]
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


def out_len(r):
    return r["k"] * r["n"] if r["coll"] == "allgather" else r["n"]


def run_server(reqs, proto="auto", sample=None, **cfg):
    """Submit all requests at once, wait, return (outputs, plans, stats).
    sample: per request None (read the whole output) or the indices to read."""
    sends = [[to_dev(x) for x in r["xs"]] for r in reqs]
    torch.cuda.synchronize()
    sample = sample or [None] * len(reqs)
    srv = Server(**cfg)
    try:
        tickets = [srv.submit(r["coll"], s, r["n"], r["dtype"], r["op"], proto=proto)
                   for r, s in zip(reqs, sends)]
        t0 = time.time()
        results = {}
        while len(results) < len(tickets):
            for i, (r, t) in enumerate(zip(reqs, tickets)):
                if t in results:
                    continue
                st, lat, plan, bufs = srv.query(t)
                if st in ("done", "failed"):
                    assert st == "done", (r["coll"], r["k"], st)
                    assert lat > 0
                    results[t] = ([read_back(bufs[q], out_len(r), r["dtype"], sample[i])
                                   for q in range(r["k"])], plan)
                    srv.release(t)          # return the buffers to the budget at once
            assert time.time() - t0 < 180, "requests did not finish"
            time.sleep(0.001)
        outs = [results[t][0] for t in tickets]
        plans = [results[t][1] for t in tickets]
        stats = srv.stats()
    finally:
        srv.destroy()
    del sends
    return outs, plans, stats


_oracle_cache = {}


def oracle_for(r, plan, slots=SMALL_SLOTS):
    """The oracle's outputs for request r under `plan` (cached per request and
    plan: the same request recurs across modes and protocols)."""
    key = (id(r), plan["proto"], plan["nchannels"], plan["chunkSteps"],
           None if slots is None else tuple(sorted(slots.items())))
    if key in _oracle_cache:
        return _oracle_cache[key]
    dt, C, cs = r["dtype"], plan["nchannels"], plan["chunkSteps"]
    if r["coll"] == "allgather":
        want = oracle.all_gather(r["xs"], C, chunk_for(plan["proto"], dt, slots, cs, True))
    else:
        ch = chunk_for(plan["proto"], dt, slots, cs)
        if r["coll"] == "allreduce":
            want = oracle.all_reduce(r["xs"], dt, r["op"], C, ch)
        else:
            want = oracle.reduce_scatter(r["xs"], dt, r["op"], C, ch)
    _oracle_cache[key] = want
    return want


CFG = dict(max_ranks=16, mem_budget=512 << 20, big_gang_channels=4, small_gangs=4,
           big_threshold=256 << 10, slot_bytes=SMALL_SLOTS, idle_timeout_sec=20.0)

_reqs = {}


def requests(name):
    """The request sets, built once per session (their oracle results are cached)."""
    if name not in _reqs:
        _reqs[name] = {"mix": lambda: make_requests(5, 40, 16, 1024, 2 << 20),
                       "budget": lambda: make_requests(9, 24, 16, 256 << 10, 1 << 20),
                       "plain": lambda: make_requests(13, 20, 16, 1024, 4 << 20)}[name]()
    return _reqs[name]


def wanted_proto(plan_proto, asked):
    """The protocol a request must run with: the one asked for, and Auto runs
    the direct protocol."""
    return ("direct" if asked == "auto" else asked) == plan_proto


@pytest.mark.parametrize("mode,proto", BATCHING)
def test_serving_results_exact_and_same_alone(mode, proto):
    reqs = requests("mix")
    outs, plans, stats = run_server(reqs, proto=proto, mode=mode, **CFG)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["maxInflightBytes"] <= CFG["mem_budget"]
    assert any(p["nchannels"] > 1 for p in plans)   # large requests spread over several channels
    for r, o, p in zip(reqs, outs, plans):
        assert wanted_proto(p["proto"], proto), p
        want = oracle_for(r, p)
        for q in range(r["k"]):
            assert_same(o[q], want[q], f"{proto} {r['coll']} k={r['k']} n={r['n']} rank {q}")
    # the same requests alone, each on a fresh server, give the same bits
    for i in (0, 7, 19, 33):
        o1, p1, _ = run_server([reqs[i]], proto=proto, mode=mode, **CFG)
        assert p1[0] == plans[i]
        for q in range(reqs[i]["k"]):
            assert_same(o1[0][q], outs[i][q], f"{proto} request {i} alone vs in the mix, rank {q}")


@pytest.mark.parametrize("mode,proto", BATCHING)
def test_serving_respects_memory_budget(mode, proto):
    reqs = requests("budget")
    budget = 40 << 20
    cfg = dict(CFG, mem_budget=budget)
    outs, plans, stats = run_server(reqs, proto=proto, mode=mode, **cfg)
    assert stats["completed"] == len(reqs)
    assert 0 < stats["maxInflightBytes"] <= budget
    for r, o, p in zip(reqs[:6], outs[:6], plans[:6]):
        want = oracle_for(r, p)
        for q in range(r["k"]):
            assert_same(o[q], want[q], f"{proto} budget {r['coll']} k={r['k']} rank {q}")


@pytest.mark.parametrize("proto", PROTOS)
def test_plain_mode_exact(proto):
    reqs = requests("plain")
    outs, plans, stats = run_server(reqs, proto=proto, mode="plain", **CFG)
    assert stats["completed"] == len(reqs)
    for r, o, p in zip(reqs, outs, plans):
        assert wanted_proto(p["proto"], proto), p
        want = oracle_for(r, p)
        for q in range(r["k"]):
            assert_same(o[q], want[q], f"{proto} plain {r['coll']} k={r['k']} rank {q}")


@pytest.mark.parametrize("proto", PROTOS)
def test_streams_and_plain_give_the_same_bits(proto):
    """Plans depend on the request alone: the lanes of the streams mode and
    one launch per request produce identical results."""
    reqs = requests("plain")
    o1, p1, _ = run_server(reqs, proto=proto, mode="streams", **CFG)
    o2, p2, _ = run_server(reqs, proto=proto, mode="plain", **CFG)
    assert p1 == p2
    for i in range(len(reqs)):
        for q in range(reqs[i]["k"]):
            assert_same(o1[i][q], o2[i][q], f"{proto} request {i} rank {q}")


def test_tiles_and_plain_give_the_same_bits():
    """The tile kernel plans like one launch per request, so the two give
    identical results."""
    reqs = requests("plain")
    o1, p1, _ = run_server(reqs, proto="auto", mode="tiles", **CFG)
    o2, p2, _ = run_server(reqs, proto="auto", mode="plain", **CFG)
    assert p1 == p2
    for i in range(len(reqs)):
        for q in range(reqs[i]["k"]):
            assert_same(o1[i][q], o2[i][q], f"tiles request {i} rank {q}")


def test_tiles_refuses_fifo_protocols():
    from paper_2507_04786_b300 import VcommError
    r = requests("plain")[0]
    s = [to_dev(x) for x in r["xs"]]
    srv = Server(mode="tiles", **{k: v for k, v in CFG.items() if k != "slot_bytes"})
    try:
        for proto in ("simple", "ll", "ll128"):
            with pytest.raises(VcommError):
                srv.submit(r["coll"], s, r["n"], r["dtype"], r["op"], proto=proto)
    finally:
        srv.destroy()


def test_tiles_kernel_restarts_after_idle():
    """The tile kernel returns after its idle timeout; later requests start it
    again and give the same bits as before."""
    reqs = requests("mix")[:6]
    sends = [[to_dev(x) for x in r["xs"]] for r in reqs]
    torch.cuda.synchronize()
    cfg = dict(CFG, idle_timeout_sec=0.2)
    srv = Server(mode="tiles", **cfg)
    try:
        got = []
        for rnd in range(3):
            tickets = [srv.submit(r["coll"], s, r["n"], r["dtype"], r["op"]) for r, s in zip(reqs, sends)]
            outs = []
            for r, t in zip(reqs, tickets):
                t0 = time.time()
                while srv.query(t)[0] not in ("done", "failed"):
                    assert time.time() - t0 < 30
                    time.sleep(0.001)
                st, lat, plan, bufs = srv.query(t)
                assert st == "done"
                outs.append(([read_back(bufs[q], out_len(r), r["dtype"]) for q in range(r["k"])], plan))
                srv.release(t)
            got.append(outs)
            time.sleep(0.6)        # longer than the idle timeout: the kernel returns
        for rnd in (1, 2):
            for i, r in enumerate(reqs):
                assert got[rnd][i][1] == got[0][i][1]
                for q in range(r["k"]):
                    assert_same(got[rnd][i][0][q], got[0][i][0][q], f"round {rnd} request {i} rank {q}")
        for i, r in enumerate(reqs):
            want = oracle_for(r, got[0][i][1])
            for q in range(r["k"]):
                assert_same(got[0][i][0][q], want[q], f"request {i} rank {q}")
    finally:
        srv.destroy()


# ------------------------------------------------------------ the largest requests

LARGE = [  # (collective, vranks, dtype, per-rank bytes S = the larger buffer)
    ("allreduce", 16, "fp32", 128 << 20),
    ("reducescatter", 13, "bf16", 64 << 20),
    ("allgather", 16, "fp32", 128 << 20),
    ("allreduce", 2, "bf16", 96 << 20),
]


@pytest.fixture(scope="module")
def large_requests():
    reqs = []
    for i, (coll, k, dt, S) in enumerate(LARGE):
        es = 4 if dt == "fp32" else 2
        n = S // es if coll == "allreduce" else S // es // k
        nin = k * n if coll == "reducescatter" else n
        xs = inputs.workload(4000 + i, k, nin, dt, "normal")
        reqs.append(dict(coll=coll, k=k, dtype=dt, n=n, xs=xs, op="sum"))
    g = np.random.default_rng(17)
    sample = []
    for r in reqs:
        m = out_len(r)
        sample.append(np.unique(np.concatenate([g.integers(0, m, 4000), [0, 1, m // 2, m - 1]])))
    return reqs, sample


SERVE_SLOTS = {"simple": 256 << 10, "ll": 32 << 10, "ll128": 300 << 10}   # the server's defaults


def sampled_want(r, plan, idx, q):
    """Oracle values of rank q's output at `idx`, one element at a time."""
    dt = r["dtype"]
    if r["coll"] == "allgather":                 # block b of every output is rank b's input
        n = r["n"]
        return np.array([r["xs"][i // n][i % n] for i in idx], dtype=r["xs"][0].dtype)
    if r["coll"] == "reducescatter":
        return oracle.reduce_scatter_points(r["xs"], q, idx, dt, r["op"])
    ch = chunk_for(plan["proto"], dt, SERVE_SLOTS, plan["chunkSteps"])
    return oracle.all_reduce_points(r["xs"], idx, dt, r["op"], plan["nchannels"], ch, "ring")


@pytest.mark.parametrize("mode,proto", [(m, p) for m in MODES for p in ("simple", "ll128", "auto")] +
                         [("tiles", "auto")])
def test_largest_requests_sampled(large_requests, mode, proto):
    """Requests at the top of the served size range (up to 16 vranks x 128 MiB)
    with the server's default FIFO slots, served together: sampled elements of
    three ranks' outputs equal the oracle's one-element replay for the
    reported plan, and every rank of an AllReduce / AllGather holds the same
    sampled values."""
    reqs, sample = large_requests
    cfg = dict(CFG, mem_budget=16 << 30, big_threshold=4 << 20, slot_bytes=SERVE_SLOTS,
               big_gang_channels=0, small_gangs=2)
    outs, plans, stats = run_server(reqs, proto=proto, sample=sample, mode=mode, **cfg)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    for r, o, p, idx in zip(reqs, outs, plans, sample):
        assert wanted_proto(p["proto"], proto), p
        same = r["coll"] != "reducescatter"
        want = None
        for q in sorted({0, r["k"] // 2, r["k"] - 1}):
            if want is None or not same:
                want = sampled_want(r, p, idx, q)
            assert_same(o[q], want, f"{mode} {proto} {r['coll']} k={r['k']} rank {q}")
        if same:
            for q in range(1, r["k"]):
                assert_same(o[q], o[0], f"{mode} {proto} {r['coll']} rank {q} vs 0")
