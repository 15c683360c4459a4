"""FIFO slot counts other than the default 8 (nsteps = 2, 3, 5, 64).

A FIFO worker keeps the slot index of each of its connections as a counter
that wraps at nsteps, started from the position earlier calls left in the
connection's head / tail counters.  A run of calls on one communicator, with
sizes that leave those positions at different slots, crosses the wrap at
every phase of the counter, on the ring (one receive and one send
connection per worker) and on the tree (two of each on inner nodes, whose
positions differ).  Every result must equal the oracle's for its plan, for
each of the paper's protocols; the slot count does not enter the result.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K, C = 5, 2

# (algorithm, collective, elements per rank (per block for ReduceScatter /
# AllGather), dtype, op, root)
CALLS = [
    ("ring", "allreduce", 3001, "fp32", "sum", 0),
    ("tree", "allreduce", 7001, "bf16", "sum", 0),
    ("ring", "reducescatter", 1501, "fp16", "sum", 0),
    ("ring", "allgather", 2003, "int32", None, 0),
    ("ring", "allreduce", 4099, "int32", "max", 0),
    ("tree", "allreduce", 2500, "fp32", "max", 0),
    ("ring", "broadcast", 5003, "fp16", None, 2),
    ("ring", "reduce", 3333, "fp32", "sum", 3),
    ("ring", "allreduce", 17, "bf16", "sum", 0),
]


def data(seed, k, n, dtype):
    if dtype == "int32":
        return inputs.workload(seed, k, n, dtype, "int", lo=-2 ** 20, hi=2 ** 20)
    return inputs.workload(seed, k, n, dtype, "normal")


def run_call(c, i, algo, coll, n, dtype, op, root, proto):
    m = K * n if coll == "reducescatter" else n
    xs = data(500 + 31 * i, K, m, dtype)
    s = [to_dev(x) for x in xs]
    outn = K * n if coll == "allgather" else n
    d = [torch.full((outn,), 7, dtype=s[0].dtype, device="cuda") for _ in range(K)]
    if coll == "allreduce":
        c.all_reduce(s, d, op=op, algo=algo, proto=proto)
    elif coll == "reducescatter":
        c.reduce_scatter(s, d, op=op, algo=algo, proto=proto)
    elif coll == "allgather":
        c.all_gather(s, d, algo=algo, proto=proto)
    elif coll == "broadcast":
        c.broadcast(s, d, root=root, algo=algo, proto=proto)
    else:
        d = [t if r == root else None for r, t in enumerate(d)]
        c.reduce(s, d, op=op, root=root, algo=algo, proto=proto)
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    ch = chunk_for(proto, dtype, SMALL_SLOTS)
    if coll == "allreduce":
        want = oracle.all_reduce(xs, dtype, op, C, ch, algo)
    elif coll == "reducescatter":
        want = oracle.reduce_scatter(xs, dtype, op, C, ch)
    elif coll == "allgather":
        want = [np.concatenate(xs)] * K
    elif coll == "broadcast":
        want = [xs[root]] * K
    else:
        want = [None] * K
        want[root] = oracle.reduce(xs, dtype, op, root, C, ch)
    for r in range(K):
        if want[r] is not None:
            assert_same(to_np(d[r], dtype), want[r], f"call {i} {algo} {coll} {dtype} rank {r}")


@pytest.mark.parametrize("nsteps", [2, 3, 5, 64])
@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
def test_calls_in_a_row_cross_the_slot_wrap(nsteps, proto):
    c = Comm(K, C, slot_bytes=SMALL_SLOTS, nsteps=nsteps, timeout_sec=10.0)
    c.set_plan(nchannels=C, chunk_steps=1)
    for rep in range(2):   # the second pass starts from the positions the first left
        for i, call in enumerate(CALLS):
            run_call(c, i + rep * len(CALLS), *call, proto)
    c.destroy()
