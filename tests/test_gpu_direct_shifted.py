"""ReduceScatter and AllGather with the direct protocol on 16-byte aligned
buffers whose blocks are not whole 16-byte units (recvcount / sendcount x
size not a multiple of 16): block b starts (b n size) mod 16 bytes into an
aligned unit, and the kernels cut each misaligned 16-byte piece out of two
aligned loads.  Every element is compared with the oracle (ReduceScatter: the
ring fold order of each block; AllGather: the plain definition), for single
calls and for a group, including the last units whose second aligned load
would pass the end of a buffer, and blocks shorter than one unit.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, group, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20}), "int8": ("int", {"lo": -100, "hi": 100}),
        "fp64": ("normal", {})}
ESZ = {"fp32": 4, "bf16": 2, "fp16": 2, "int32": 4, "int8": 1, "fp64": 8}

# (vranks, elements per block) with n x size not a multiple of 16 for every type
CASES = [(3, 1), (3, 5), (5, 1001), (12, 7001), (16, 333), (7, 65539), (2, 3), (16, 131075)]


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


@pytest.mark.parametrize("k,n", CASES)
@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max"), ("int32", "sum"),
                                      ("int8", "sum"), ("fp64", "min")])
def test_reduce_scatter_shifted(k, n, dtype, op):
    xs = data(100 * k + n, k, k * n, dtype)
    c = Comm(k, 4, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    c.set_plan(nchannels=4, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.full((n,), 3, dtype=s[0].dtype, device="cuda") for _ in range(k)]
    c.reduce_scatter(s, d, op=op, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    want = oracle.reduce_scatter(xs, dtype, op, 4, chunk_for("simple", dtype, SMALL_SLOTS, 1))
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"RS k={k} n={n} {dtype} rank {r}")
    c.destroy()


@pytest.mark.parametrize("k,n", CASES)
@pytest.mark.parametrize("dtype", ["fp32", "bf16", "int8", "fp64"])
def test_all_gather_shifted(k, n, dtype):
    xs = data(200 * k + n, k, n, dtype)
    c = Comm(k, 4, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    s = [to_dev(x) for x in xs]
    d = [torch.full((k * n,), 5, dtype=s[0].dtype, device="cuda") for _ in range(k)]
    c.all_gather(s, d, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    whole = np.concatenate(xs)
    for r in range(k):
        assert_same(to_np(d[r], dtype), whole, f"AG k={k} n={n} {dtype} rank {r}")
    c.destroy()


def test_group_of_shifted_calls():
    """ReduceScatter and AllGather calls with whole and partial units in one
    group (one launch of the tile engine: staged windows for the shifted
    ReduceScatter blocks, the register path for the shifted AllGather)."""
    k = 6
    c = Comm(k, 4, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    c.set_plan(nchannels=4, chunk_steps=1)
    calls = []
    for i, (n, dt) in enumerate([(1001, "fp32"), (1024, "fp32"), (77, "bf16"), (4099, "bf16"), (5, "int32")]):
        xs = data(300 + i, k, k * n, dt)
        s = [to_dev(x) for x in xs]
        d = [torch.empty((n,), dtype=s[0].dtype, device="cuda") for _ in range(k)]
        g = data(400 + i, k, n, dt)
        gs = [to_dev(x) for x in g]
        gd = [torch.empty((k * n,), dtype=gs[0].dtype, device="cuda") for _ in range(k)]
        calls.append((n, dt, xs, s, d, g, gs, gd))
    with group():
        for n, dt, xs, s, d, g, gs, gd in calls:
            c.reduce_scatter(s, d, op="sum", algo="ring", proto="direct")
            c.all_gather(gs, gd, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    for n, dt, xs, s, d, g, gs, gd in calls:
        want = oracle.reduce_scatter(xs, dt, "sum", 4, chunk_for("simple", dt, SMALL_SLOTS, 1))
        for r in range(k):
            assert_same(to_np(d[r], dt), want[r], f"group RS n={n} {dt} rank {r}")
            assert_same(to_np(gd[r], dt), np.concatenate(g), f"group AG n={n} {dt} rank {r}")
    c.destroy()
