"""GPU parity of the direct reducing collectives staged through shared
memory (bulk asynchronous copies, kDirectReduceStaged) against the CPU
oracle, bit-exact.

The staged kernel takes aligned AllReduce calls on 2..16 vranks (fp64: up to
8) and ReduceScatter / Reduce calls on 2..4 vranks from
VCOMM_STAGED_MIN_BYTES per rank (read when a communicator is created).  These tests create their communicators with that threshold at 16
bytes, so sizes the oracle replays in seconds already run staged and span
many tiles, several CTAs, segments that straddle tiles, a ragged last tile
and an element tail, with two stages (up to 4 vranks) and three; small
Simple slots make segments short.  Its results must equal the oracle's ring
results for Simple's chunk, the register kernel's bit for bit, and a Simple
call's.  Beyond the rule's limits the register kernel runs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BITS = {"int8": (8, True), "uint8": (8, False), "int32": (32, True), "uint32": (32, False),
        "int64": (64, True), "uint64": (64, False)}
TORCH_INT = {1: torch.int8, 2: torch.int16, 4: torch.int32, 8: torch.int64}

_comms = {}


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    assert torch.cuda.is_available()
    yield
    for c in _comms.values():
        c.destroy()
    _comms.clear()


def make_comm(k, C, min_bytes):
    old = os.environ.get("VCOMM_STAGED_MIN_BYTES")
    os.environ["VCOMM_STAGED_MIN_BYTES"] = str(min_bytes)
    try:
        return Comm(k, C, slot_bytes=SMALL_SLOTS, timeout_sec=10.0)
    finally:
        if old is None:
            del os.environ["VCOMM_STAGED_MIN_BYTES"]
        else:
            os.environ["VCOMM_STAGED_MIN_BYTES"] = old


def get_comm(k, C, staged=True):
    key = (k, C, staged)
    if key not in _comms:
        _comms[key] = make_comm(k, C, 16 if staged else 1 << 62)
    return _comms[key]


def data(seed, k, n, dtype, op="sum"):
    if dtype in BITS:
        bits, signed = BITS[dtype]
        lo, hi = (-2 ** (bits - 1), 2 ** (bits - 1) - 1) if signed else (0, 2 ** bits - 1)
        return inputs.workload(seed, k, n, dtype, "int", lo=lo, hi=hi)
    return inputs.workload(seed, k, n, dtype, "pow2" if op == "prod" else "normal")


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


def bits_of(t):
    return t.view(TORCH_INT[t.element_size()])


CASES = [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max"), ("int32", "sum"), ("fp32", "avg"),
         ("fp64", "prod"), ("int8", "min"), ("uint64", "sum"), ("bf16", "avg"), ("uint8", "max")]


@pytest.mark.parametrize("dtype,op", CASES)
@pytest.mark.parametrize("k,C,steps", [(2, 1, 1), (3, 3, 2), (4, 2, 1), (5, 2, 2), (8, 8, 1),
                                       (16, 3, 3), (33, 2, 1)])
def test_staged_allreduce(dtype, op, k, C, steps):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=steps)
    sizes = (5, 1000, 8195, 100003) if k <= 16 else (37, 8195, 30011)
    for n in sizes:
        xs = data(n + 3 * k + len(op), k, n, dtype, op)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo="ring", proto="direct")
        finish(c)
        p = c.last_plan()
        assert (p["algo"], p["proto"], p["nchannels"]) == ("ring", "direct", C)
        want = oracle.all_reduce(xs, dtype, op, C, chunk_for("simple", dtype, SMALL_SLOTS, steps))
        for r in sorted({0, k // 2, k - 1}):
            assert_same(to_np(d[r], dtype), want[r], f"n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "int64"])
@pytest.mark.parametrize("k,C", [(4, 2), (8, 37), (16, 5)])
def test_equals_register_kernel_and_simple(dtype, k, C):
    """The same call through the staged kernel, the register kernel and the
    Simple FIFO protocol: three identical results."""
    cs, cr = get_comm(k, C, True), get_comm(k, C, False)
    for c in (cs, cr):
        c.set_plan(nchannels=C, chunk_steps=1)
    n = (3 << 20) // 4 + 13                      # ~3 MiB per rank and an element tail
    xs = data(77 + k, k, n, dtype)
    s = [to_dev(x) for x in xs]
    d1, d2, d3 = ([torch.empty_like(t) for t in s] for _ in range(3))
    cs.all_reduce(s, d1, algo="ring", proto="direct")
    cr.all_reduce(s, d2, algo="ring", proto="direct")
    cr.all_reduce(s, d3, algo="ring", proto="simple")
    finish(cs)
    finish(cr)
    for r in range(k):
        assert torch.equal(bits_of(d1[r]), bits_of(d2[r])), f"staged vs register rank {r}"
        assert torch.equal(bits_of(d1[r]), bits_of(d3[r])), f"staged vs simple rank {r}"
    for c in (cs, cr):
        c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("int32", "max"),
                                      ("fp16", "avg"), ("int8", "prod")])
@pytest.mark.parametrize("k", [2, 3, 4, 16])
def test_staged_reduce_scatter(dtype, op, k):
    """ReduceScatter blocks of whole 16-byte units run staged on up to 4
    vranks (tiles never straddle blocks); other block sizes and 16 vranks
    take the register kernel."""
    c = get_comm(k, 2)
    c.set_plan(nchannels=2, chunk_steps=1)
    for m in (16, 4096, 50000, 777):              # 777: not whole units for 2- and 4-byte types
        xs = data(m + 11 * k + len(op), k, k * m, dtype, op)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.reduce_scatter(s, d, op=op, algo="ring", proto="direct")
        finish(c)
        want = oracle.reduce_scatter(xs, dtype, op, 2, chunk_for("simple", dtype, SMALL_SLOTS, 1))
        for r in sorted({0, k // 2, k - 1}):
            assert_same(to_np(d[r], dtype), want[r], f"m={m} rank {r}")
    m = 20000                                      # in place: recvbuf r is block r of sendbuf r
    xs = data(9 * k, k, k * m, dtype, op)
    s = [to_dev(x) for x in xs]
    c.reduce_scatter(s, [t[r * m:(r + 1) * m] for r, t in enumerate(s)], op=op, algo="ring",
                     proto="direct")
    finish(c)
    want = oracle.reduce_scatter(xs, dtype, op, 2, chunk_for("simple", dtype, SMALL_SLOTS, 1))
    for r in range(k):
        assert_same(to_np(s[r][r * m:(r + 1) * m], dtype), want[r], f"in place rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "max"), ("int32", "sum"),
                                      ("fp64", "min")])
@pytest.mark.parametrize("k,root", [(2, 1), (3, 0), (4, 3), (16, 0)])
def test_staged_reduce(dtype, op, k, root):
    c = get_comm(k, 1)
    c.set_plan(nchannels=1, chunk_steps=1)
    for n in (5, 2049, 30011, 100003):
        xs = data(n + 7 * root, k, n, dtype, op)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(s[0]) if r == root else None for r in range(k)]
        c.reduce(s, d, op=op, root=root, algo="ring", proto="direct")
        finish(c)
        want = oracle.reduce(xs, dtype, op, root, 1, chunk_for("simple", dtype, SMALL_SLOTS, 1))
        assert_same(to_np(d[root], dtype), want, f"n={n}")
        d = [s[root] if r == root else None for r in range(k)]     # the root in place
        c.reduce(s, d, op=op, root=root, algo="ring", proto="direct")
        finish(c)
        assert_same(to_np(s[root], dtype), want, f"in place n={n}")
    c.clear_plan()


def test_in_place_and_unaligned_fallback():
    """In place (recvbuf = sendbuf) runs staged; a view at an odd element
    offset is not 16-byte aligned and takes the element-wise kernel; both
    equal the oracle."""
    k, C, n = 6, 3, 50021
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    xs = data(31, k, n, "fp32")
    want = oracle.all_reduce(xs, "fp32", "sum", C, chunk_for("simple", "fp32", SMALL_SLOTS, 1))
    s = [to_dev(x) for x in xs]
    c.all_reduce(s, s, op="sum", algo="ring", proto="direct")
    finish(c)
    for r in range(k):
        assert_same(to_np(s[r], "fp32"), want[r], f"in place rank {r}")
    s = [to_dev(np.concatenate([x[:1], x]))[1:] for x in xs]
    d = [torch.empty(n + 1, device="cuda")[1:] for _ in range(k)]
    c.all_reduce(s, d, op="sum", algo="ring", proto="direct")
    finish(c)
    for r in range(k):
        assert_same(to_np(d[r], "fp32"), want[r], f"unaligned rank {r}")
    c.clear_plan()


def test_headline_size_default_threshold():
    """8 vranks x 256 MiB fp32 with the default threshold (staged): sampled
    elements against the oracle's one-element queries; two calls in a row
    on the same buffers give the same bits."""
    k, n, C = 8, (256 << 20) // 4, 37
    g = torch.Generator(device="cuda").manual_seed(9)
    s = [torch.randn(n, device="cuda", generator=g) for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c = Comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    c.all_reduce(s, d, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4000), [0, 1, n - 2, n - 1]]))
    t = torch.from_numpy(idx).cuda()
    full = [x.cpu().numpy() for x in s]
    want = oracle.all_reduce_points(full, idx, "fp32", "sum", C, chunk_for("simple", "fp32", None, 1))
    del full
    for r in (0, 5, 7):
        assert_same(d[r][t].cpu().numpy(), want, f"rank {r}")
    first = d[3].clone()
    c.all_reduce(s, d, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    assert torch.equal(first.view(torch.int32), d[3].view(torch.int32))
    c.destroy()


def kernels_of(c, k, n, dtype=torch.float32):
    """Names of the kernels one direct AllReduce of n elements launches."""
    prof = pytest.importorskip("torch.profiler")
    s = [torch.ones(n, device="cuda", dtype=dtype) for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    torch.cuda.synchronize()
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        c.all_reduce(s, d, algo="ring", proto="direct")
        torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    assert float(d[k - 1][-1]) == float(k)
    return [e.name for e in p.events()]


def test_threshold_and_rule_pick_the_kernel():
    """The launch list shows which kernel ran: staged at or above the
    threshold on 2..16 vranks, the register kernel below it, beyond 16
    vranks, and for fp64 beyond 8 vranks."""
    c4 = make_comm(4, 2, 1 << 20)
    large = kernels_of(c4, 4, (1 << 20) // 4)
    small = kernels_of(c4, 4, (1 << 20) // 4 - 4)
    c4.destroy()
    if not large:
        pytest.skip("the profiler recorded no CUDA kernels")
    assert any("kDirectReduceStaged" in x for x in large)
    assert not any("kDirectReduceStaged" in x for x in small)
    assert any("kDirectReduce" in x for x in small)
    c17 = make_comm(17, 1, 16)
    beyond = kernels_of(c17, 17, 100000)
    c17.destroy()
    assert not any("kDirectReduceStaged" in x for x in beyond)
    c16 = make_comm(16, 1, 16)
    f64 = kernels_of(c16, 16, 100000, torch.float64)
    f32 = kernels_of(c16, 16, 100000)
    c16.destroy()
    assert not any("kDirectReduceStaged" in x for x in f64)
    assert any("kDirectReduceStaged" in x for x in f32)
    c3 = make_comm(3, 1, 16)
    prof = pytest.importorskip("torch.profiler")
    s = [torch.ones(3 * 4096, device="cuda") for _ in range(3)]
    d = [torch.empty(4096, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        c3.reduce_scatter(s, d, algo="ring", proto="direct")
        torch.cuda.synchronize()
    assert c3.async_error() == "vSuccess" and float(d[2][-1]) == 3.0
    c3.destroy()
    assert any("kDirectReduceStaged" in e.name for e in p.events())
