"""Every element, at the sizes where the chunk and loop structure is in full
swing: several loops of full FIFO chunks per channel.

* The protocol sweep's AllReduce on 8 vranks at 64 MiB per vrank, fp32 and
  bf16 N(0,1), with Simple, LL128 and the direct protocol (37 channels): every
  element of every rank against the oracle's full replay of the plan.
* The tree / ring workload at 4, 16 and 64 MiB per vrank on 8 and 16 vranks:
  tree AllReduce and ring ReduceScatter, AllGather, Broadcast (root 0) and
  Reduce (root 0); fp16 U[-1, 1] and int32 U[-2^20, 2^20]; sum and max; with
  the Simple protocol and with Auto.  fp16 sums are compared with the oracle's
  replay of the schedule; int32 sums (two's-complement wraparound) and every
  max are order-free, so they are compared with a brute-force elementwise
  fold; copies with the plain definition.

The oracle runs in host threads (it releases the interpreter lock), one per
independent replay.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import bench
import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MiB = 1 << 20


def _finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


# ---------------------------------------------------------------- 8 x 64 MiB ring AllReduce

@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_allreduce_8vr_64MiB_every_element(dtype):
    k, C, S = 8, 37, 64 * MiB
    es = 4 if dtype == "fp32" else 2
    n = S // es
    xs = inputs.workload(21, k, n, dtype, "normal")
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c = Comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    thr = bench.oracle_threads(C)
    want = {}
    for proto in ("simple", "ll128"):
        want[proto] = bench.oracle_all_reduce(xs, dtype, "sum", C, chunk_for(proto, dtype, None, 1), thr)
    want["direct"] = want["simple"]                    # the direct protocol folds Simple's segments
    for proto in ("simple", "ll128", "direct"):
        for t in d:
            t.fill_(7)
        c.all_reduce(s, d, op="sum", algo="ring", proto=proto)
        _finish(c)
        p = c.last_plan()
        assert p["proto"] == proto and p["nchannels"] == C, p
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[proto][r], f"{proto} {dtype} rank {r}")
    c.destroy()


# ---------------------------------------------------------------- the tree / ring workload

def _vals(seed, k, n, dtype):
    if dtype == "fp16":
        return inputs.workload(seed, k, n, "fp16", "uniform")
    return inputs.workload(seed, k, n, "int32", "int", lo=-2 ** 20, hi=2 ** 20)


def _brute(xs, op):
    """Order-free fold over the ranks: int32 sums wrap, max elementwise."""
    st = np.stack(xs)
    if op == "max":
        return np.maximum.reduce(st, axis=0)
    assert st.dtype == np.int32
    return np.sum(st, axis=0, dtype=np.int32)


def _same_max(got, want, what):
    """max of floats: equal values, and equal bits except where the result is
    a zero (+0 and -0 compare equal; the schedule order decides the sign)."""
    nz = want != 0
    assert np.array_equal(got[~nz] == 0, np.ones((~nz).sum(), bool)), what
    assert_same(got[nz], want[nz], what)


SIZES = [4 * MiB, 16 * MiB, 64 * MiB]


@pytest.mark.parametrize("dtype", ["fp16", "int32"])
@pytest.mark.parametrize("S", SIZES, ids=lambda s: f"{s >> 20}MiB")
@pytest.mark.parametrize("k", [8, 16])
def test_tree_and_ring_collectives_every_element(k, S, dtype):
    es = 2 if dtype == "fp16" else 4
    C = 16 if k == 8 else 8
    n = S // es                       # S = the larger per-rank buffer
    m = n // k
    xs = _vals(3000 + k + S // MiB, k, n, dtype)
    protos_ring = ("simple", "auto")
    protos_tree = ("simple", "ll128") if S == 4 * MiB else ("simple",)

    # expected values first: order-free ones by brute force, fp16 sums by the
    # oracle's replay of the pinned plan (C channels, one slot per chunk)
    full = {op: _brute(xs, op) for op in (("sum", "max") if dtype == "int32" else ("max",))}
    replay = {}
    if dtype == "fp16":
        jobs = {("allreduce", pr): (oracle.all_reduce, (xs, dtype, "sum", C, chunk_for(pr, dtype, None, 1),
                                                        "tree")) for pr in protos_tree}
        # the ring ReduceScatter's fold order of block b and the Reduce chain's
        # order do not depend on channels or chunk: one replay serves every plan
        ch = chunk_for("simple", dtype, None, 1)
        jobs[("reducescatter",)] = (oracle.reduce_scatter, (xs, dtype, "sum", C, ch))
        jobs[("reduce",)] = (oracle.reduce, (xs, dtype, "sum", 0, C, ch))
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = {key: ex.submit(f, *a) for key, (f, a) in jobs.items()}
            replay = {key: f.result() for key, f in futs.items()}

    def expected(coll, op, proto):
        if op == "sum" and dtype == "fp16":
            if coll == "allreduce":
                return replay[("allreduce", proto)]
            if coll == "reducescatter":
                return replay[("reducescatter",)]
            return [replay[("reduce",)]]
        ref = full[op]
        return {"allreduce": [ref] * k, "reducescatter": [ref[b * m:(b + 1) * m] for b in range(k)],
                "reduce": [ref]}[coll]

    s = [to_dev(x) for x in xs]
    c = Comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)

    def check(coll, op, proto, outs, algo):
        torch.cuda.synchronize()
        assert c.async_error() == "vSuccess"
        p = c.last_plan()
        assert p["nchannels"] == C and p["chunkSteps"] == 1 and p["algo"] == algo, p
        what = f"{coll} {op} {proto} k={k} {S >> 20}MiB {dtype} plan {p}"
        if coll == "allgather":
            whole = np.concatenate([x[:m] for x in xs])
            wants = [whole] * k
        elif coll == "broadcast":
            wants = [xs[0]] * k
        else:
            wants = expected(coll, op, proto)
        for r, w in enumerate(wants):
            got = to_np(outs[r], dtype)
            if op == "max" and dtype == "fp16":
                _same_max(got, w, f"{what} rank {r}")
            else:
                assert_same(got, w, f"{what} rank {r}")

    for op in ("sum", "max"):
        for proto in protos_tree:
            d = [torch.empty_like(t) for t in s]
            c.all_reduce(s, d, op=op, algo="tree", proto=proto)
            check("allreduce", op, proto, d, "tree")
        for proto in protos_ring:
            d = [torch.empty(m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
            c.reduce_scatter(s, d, op=op, algo="ring", proto=proto)
            check("reducescatter", op, proto, d, "ring")
            d = [torch.empty_like(s[0])] + [None] * (k - 1)
            c.reduce(s, d, op=op, root=0, algo="ring", proto=proto)
            check("reduce", op, proto, d, "ring")
    for proto in protos_ring:
        d = [torch.empty(n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather([t[:m] for t in s], d, algo="ring", proto=proto)
        check("allgather", None, proto, d, "ring")
        d = [torch.empty_like(t) for t in s]
        c.broadcast(s, d, root=0, algo="ring", proto=proto)
        check("broadcast", None, proto, d, "ring")
    c.destroy()
