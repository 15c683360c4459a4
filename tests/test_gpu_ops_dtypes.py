"""GPU parity of the element types and reductions beyond sum / max on
fp32 / fp16 / bf16 / int32: int8, uint8, uint32, int64, uint64, fp64 and prod,
min, avg, for every protocol (Simple, LL, LL128, cluster, direct), ring and
tree, bit-exact against the oracle.

Integers cover their full range (sums and products wrap); floats are N(0,1)
for sum / min / max / avg and +-2^e for prod.  avg divides the completed
value once (the oracle's reading); sizes are ragged and span several FIFO
steps with small slots.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, group, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TYPES = ["int8", "uint8", "int32", "uint32", "int64", "uint64", "fp16", "bf16", "fp32", "fp64"]
OPS = ["sum", "prod", "max", "min", "avg"]
BITS = {"int8": (8, True), "uint8": (8, False), "int32": (32, True), "uint32": (32, False),
        "int64": (64, True), "uint64": (64, False)}

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
        _comms[(k, C)] = Comm(k, C, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    return _comms[(k, C)]


def data(seed, k, n, dtype, op):
    if dtype in BITS:
        bits, signed = BITS[dtype]
        lo, hi = (-2 ** (bits - 1), 2 ** (bits - 1) - 1) if signed else (0, 2 ** bits - 1)
        return inputs.workload(seed, k, n, dtype, "int", lo=lo, hi=hi)
    return inputs.workload(seed, k, n, dtype, "pow2" if op == "prod" else "normal")


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


CASES = [(proto, algo) for proto in ("simple", "ll", "ll128", "cluster", "direct")
         for algo in (("ring", "tree") if proto != "direct" else ("ring",))]


@pytest.mark.parametrize("proto,algo", CASES)
@pytest.mark.parametrize("dtype", TYPES)
@pytest.mark.parametrize("op", OPS)
def test_allreduce(proto, algo, dtype, op):
    k, C = 5, 2
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    for n in (1, 1003, 20011):
        xs = data(n + 17 * len(dtype) + len(op), k, n, dtype, op)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo=algo, proto=proto)
        finish(c)
        p = c.last_plan()
        want = oracle.all_reduce(xs, dtype, op, p["nchannels"],
                                 chunk_for(p["proto"], dtype, SMALL_SLOTS, p["chunkSteps"]), p["algo"])
        for r in (0, 2, k - 1):
            assert_same(to_np(d[r], dtype), want[r], f"{proto}/{algo} {dtype} {op} n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128", "cluster", "direct"])
@pytest.mark.parametrize("dtype", ["int8", "uint32", "int64", "fp64", "bf16"])
@pytest.mark.parametrize("op", ["prod", "min", "avg"])
def test_reduce_scatter_and_reduce(proto, dtype, op):
    k, C = 4, 3
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    m = 2049
    xs = data(5 + m, k, k * m, dtype, op)
    s = [to_dev(x) for x in xs]
    d = [torch.empty(m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
    c.reduce_scatter(s, d, op=op, algo="ring", proto=proto)
    finish(c)
    ch = chunk_for(proto, dtype, SMALL_SLOTS, 1)
    want = oracle.reduce_scatter(xs, dtype, op, C, ch)
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"RS {proto} {dtype} {op} rank {r}")
    ys = [x[:m].copy() for x in xs]
    t = [to_dev(y) for y in ys]
    root = 2
    out = [torch.empty_like(t[0]) if r == root else None for r in range(k)]
    c.reduce(t, out, op=op, root=root, algo="ring", proto=proto)
    finish(c)
    assert_same(to_np(out[root], dtype), oracle.reduce(ys, dtype, op, root, C, ch),
                f"Reduce {proto} {dtype} {op}")
    c.clear_plan()


@pytest.mark.parametrize("proto", ["simple", "ll128", "direct"])
@pytest.mark.parametrize("dtype", ["int8", "fp64", "uint64"])
def test_copies(proto, dtype):
    k, C = 3, 2
    c = get_comm(k, C)
    for n in (1, 999, 8191):
        xs = data(n, k, n, dtype, "sum")
        s = [to_dev(x) for x in xs]
        d = [torch.empty(k * n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto=proto)
        b = [torch.empty_like(t) for t in s]
        c.broadcast(s, b, root=1, algo="ring", proto=proto)
        finish(c)
        for r in range(k):
            assert_same(to_np(d[r], dtype), np.concatenate(xs), f"AG {dtype} rank {r}")
            assert_same(to_np(b[r], dtype), xs[1], f"Bcast {dtype} rank {r}")


@pytest.mark.parametrize("proto", ["simple", "ll", "direct"])
def test_mixed_group(proto):
    """A group of calls of every new type and op runs as one batch launch
    (the FIFO batch kernel or the direct batch kernels) and each result is
    the oracle's for its reported plan."""
    k = 4
    c = get_comm(k, 4)
    rng = np.random.default_rng(8)
    calls = []
    with group():
        for i in range(24):
            dtype = TYPES[i % len(TYPES)]
            op = OPS[int(rng.integers(len(OPS)))]
            n = int(rng.choice([5, 777, 4099]))
            xs = data(300 + i, k, n, dtype, op)
            s = [to_dev(x) for x in xs]
            d = [torch.empty_like(t) for t in s]
            c.all_reduce(s, d, op=op, algo="ring", proto=proto)
            calls.append((dtype, op, xs, s, d))    # keep s alive until the group has run
    finish(c)
    plans = c.group_plans()
    for (dtype, op, xs, _, d), p in zip(calls, plans):
        want = oracle.all_reduce(xs, dtype, op, p["nchannels"],
                                 chunk_for(p["proto"], dtype, SMALL_SLOTS, p["chunkSteps"]), p["algo"])
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"{proto} {dtype} {op} rank {r}")
