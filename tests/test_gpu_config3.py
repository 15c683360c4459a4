"""The tree / ring collective workload at its full size range: tree AllReduce on
8 and 16 vranks, ring ReduceScatter, AllGather, Broadcast (root 0) and Reduce
(root 0); fp16 values uniform in [-1, 1] and int32 values uniform in
[-2^20, 2^20]; sum and max; per-rank sizes 4 KiB .. 128 MiB.

Up to 1 MiB every element is compared with the oracle; at 128 MiB sampled
elements are compared with the oracle's one-element queries (and copies with
the plain definition).  Plans are the library's own (Auto) and read back.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MiB = 1 << 20
SMALL = [4096 * 4 ** i for i in range(5)]          # 4 KiB .. 1 MiB
BIG = 128 * MiB


def vals(seed, k, n, dtype):
    if dtype == "fp16":
        return inputs.workload(seed, k, n, "fp16", "uniform")
    return inputs.workload(seed, k, n, "int32", "int", lo=-2 ** 20, hi=2 ** 20)


def es(dtype):
    return 2 if dtype == "fp16" else 4


def run(c, coll, xs, dtype, op, algo, root=0):
    k = len(xs)
    s = [to_dev(x) for x in xs]
    if coll == "allreduce":
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo=algo, proto="auto")
    elif coll == "reducescatter":
        d = [torch.empty(s[0].numel() // k, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.reduce_scatter(s, d, op=op, algo="ring", proto="auto")
    elif coll == "allgather":
        d = [torch.empty(k * s[0].numel(), dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto="auto")
    elif coll == "broadcast":
        d = [torch.empty_like(t) for t in s]
        c.broadcast(s, d, root=root, algo="ring", proto="auto")
    else:
        d = [torch.empty_like(s[0]) if r == root else None for r in range(k)]
        c.reduce(s, d, op=op, root=root, algo="ring", proto="auto")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    return s, d, c.last_plan()


CASES = [("allreduce", "tree", 8, "fp16", "sum"), ("allreduce", "tree", 16, "int32", "max"),
         ("allreduce", "tree", 16, "fp16", "sum"), ("reducescatter", "ring", 8, "fp16", "sum"),
         ("reducescatter", "ring", 16, "int32", "max"), ("allgather", "ring", 8, "fp16", None),
         ("allgather", "ring", 16, "int32", None), ("broadcast", "ring", 8, "int32", None),
         ("broadcast", "ring", 16, "fp16", None), ("reduce", "ring", 8, "fp16", "sum"),
         ("reduce", "ring", 16, "int32", "max")]


@pytest.mark.parametrize("coll,algo,k,dtype,op", CASES)
def test_sizes_4KiB_to_1MiB_exact(coll, algo, k, dtype, op):
    c = Comm(k, 8)
    for S in SMALL:
        # S = the larger per-rank buffer: RS sendbuf, AG recvbuf
        n = S // es(dtype) if coll not in ("allgather",) else S // es(dtype) // k
        xs = vals(S + k, k, n, dtype)
        s, d, p = run(c, coll, xs, dtype, op, algo)
        C = p["nchannels"]
        if coll in ("allgather", "broadcast"):
            ch = chunk_for(p["proto"], dtype, None, p["chunkSteps"], byte_units=True)
            want = oracle.all_gather(xs, C, ch) if coll == "allgather" else oracle.broadcast(xs, 0, C, ch)
            for r in range(k):
                assert_same(to_np(d[r], dtype), want[r], f"{coll} {S} rank {r}")
            continue
        ch = chunk_for(p["proto"], dtype, None, p["chunkSteps"])
        if coll == "allreduce":
            want = oracle.all_reduce(xs, dtype, op, C, ch, p["algo"])
            for r in range(k):
                assert_same(to_np(d[r], dtype), want[r], f"{coll} {S} {p} rank {r}")
        elif coll == "reducescatter":
            want = oracle.reduce_scatter(xs, dtype, op, C, ch)
            for r in range(k):
                assert_same(to_np(d[r], dtype), want[r], f"{coll} {S} rank {r}")
        else:
            assert_same(to_np(d[0], dtype), oracle.reduce(xs, dtype, op, 0, C, ch), f"{coll} {S}")
    c.destroy()


BIG_CASES = [("allreduce", "tree", 16, "fp16", "sum"), ("allreduce", "tree", 8, "int32", "max"),
             ("reducescatter", "ring", 8, "fp16", "sum"), ("allgather", "ring", 8, "int32", None),
             ("broadcast", "ring", 16, "fp16", None), ("reduce", "ring", 16, "int32", "max")]


@pytest.mark.parametrize("coll,algo,k,dtype,op", BIG_CASES)
def test_128MiB_sampled(coll, algo, k, dtype, op):
    n = BIG // es(dtype) if coll != "allgather" else BIG // es(dtype) // k
    xs = vals(77 + k, k, n, dtype)
    c = Comm(k, 16)
    s, d, p = run(c, coll, xs, dtype, op, algo)
    g = np.random.default_rng(k)
    if coll == "allreduce":
        idx = np.unique(np.concatenate([g.integers(0, n, 3000), [0, n - 1]]))
        want = oracle.all_reduce_points(xs, idx, dtype, op, p["nchannels"],
                                        chunk_for(p["proto"], dtype, None, p["chunkSteps"]), p["algo"])
        t = torch.from_numpy(idx).cuda()
        for r in (0, k // 2, k - 1):
            assert_same(to_np(d[r][t], dtype), want, f"AR {p} rank {r}")
        for r in range(1, k):
            assert torch.equal(d[r].view(torch.int16 if dtype == "fp16" else torch.int32),
                               d[0].view(torch.int16 if dtype == "fp16" else torch.int32))
    elif coll == "reducescatter":
        m = n // k
        idx = np.unique(np.concatenate([g.integers(0, m, 2000), [0, m - 1]]))
        t = torch.from_numpy(idx).cuda()
        for b in (0, k - 1):
            want = oracle.reduce_scatter_points(xs, b, idx, dtype, op)
            assert_same(to_np(d[b][t], dtype), want, f"RS rank {b}")
    elif coll == "reduce":
        idx = np.unique(np.concatenate([g.integers(0, n, 3000), [0, n - 1]]))
        want = oracle.reduce_points(xs, 0, idx, dtype, op)
        assert_same(to_np(d[0][torch.from_numpy(idx).cuda()], dtype), want, "Reduce root 0")
    else:
        # copies: the plain definition on sampled positions of every rank
        idx = np.unique(np.concatenate([g.integers(0, d[0].numel(), 4000), [0, d[0].numel() - 1]]))
        t = torch.from_numpy(idx).cuda()
        whole = np.concatenate(xs) if coll == "allgather" else xs[0]
        for r in range(k):
            assert_same(to_np(d[r][t], dtype), whole[idx], f"{coll} rank {r}")
    c.destroy()
