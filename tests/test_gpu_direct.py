"""GPU parity of the direct protocol (no FIFO: each unit's ring chain folded
from the k user buffers) against the CPU oracle, bit-exact.

The direct protocol takes its segments from the Simple protocol's partition
(channels, loops, chunkCount of the Simple slot), so its expected values are
the oracle's ring results for Simple's chunk, and for one plan it must equal
a Simple call bit for bit.  Small Simple slots make modest sizes span many
loops and segments; odd element offsets exercise the unaligned path.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, VcommError, group, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}
SIZES = [1, 7, 1000, 8195, 100003]

_comms = {}


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    assert torch.cuda.is_available()
    yield
    for c in _comms.values():
        c.destroy()
    _comms.clear()


def get_comm(k, C, slots=SMALL_SLOTS):
    key = (k, C, slots is None)
    if key not in _comms:
        _comms[key] = Comm(k, C, slot_bytes=slots, timeout_sec=10.0)
    return _comms[key]


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def chunk(dtype, steps, byte_units=False):
    return chunk_for("simple", dtype, SMALL_SLOTS, steps, byte_units=byte_units)


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


def offset_views(xs, off):
    """Device copies of xs starting `off` elements into a larger buffer."""
    out = []
    for x in xs:
        t = to_dev(np.concatenate([x[:1].repeat(off), x]) if off else x)
        out.append(t[off:])
    return out


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max"),
                                      ("int32", "sum"), ("fp32", "max"), ("bf16", "max")])
@pytest.mark.parametrize("k,C,steps", [(2, 1, 1), (3, 3, 2), (5, 2, 1), (8, 8, 1), (16, 3, 3),
                                       (33, 2, 1)])
def test_ring_allreduce(dtype, op, k, C, steps):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=steps)
    for n in SIZES:
        xs = data(n + 3 * k, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo="ring", proto="direct")
        finish(c)
        p = c.last_plan()
        assert (p["algo"], p["proto"], p["nchannels"]) == ("ring", "direct", C)
        want = oracle.all_reduce(xs, dtype, op, C, chunk(dtype, steps))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"n={n} rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("k,C", [(4, 2), (8, 5)])
def test_equals_simple_for_the_same_plan(dtype, k, C):
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    n = 300007
    xs = data(91 + k, k, n, dtype)
    s = [to_dev(x) for x in xs]
    d1 = [torch.empty_like(t) for t in s]
    d2 = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d1, algo="ring", proto="simple")
    c.all_reduce(s, d2, algo="ring", proto="direct")
    finish(c)
    for r in range(k):
        assert torch.equal(d1[r].view(torch.int16 if dtype != "fp32" else torch.int32),
                           d2[r].view(torch.int16 if dtype != "fp32" else torch.int32))
    c.clear_plan()


@pytest.mark.parametrize("off", [1, 3])
def test_unaligned_and_in_place(off):
    k, C, n = 5, 3, 20011
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    xs = data(7 + off, k, n, "bf16")
    s = offset_views(xs, off)
    d = [torch.empty(n + off, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
    c.all_reduce(s, d, op="sum", algo="ring", proto="direct")
    finish(c)
    want = oracle.all_reduce(xs, "bf16", "sum", C, chunk("bf16", 1))
    for r in range(k):
        assert_same(to_np(d[r], "bf16"), want[r], f"rank {r}")
    c.all_reduce(s, s, op="sum", algo="ring", proto="direct")      # in place
    finish(c)
    for r in range(k):
        assert_same(to_np(s[r], "bf16"), want[r], f"in place rank {r}")
    c.clear_plan()


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("fp16", "sum"), ("int32", "max")])
@pytest.mark.parametrize("k", [2, 6, 16])
@pytest.mark.parametrize("off", [0, 1])
def test_reduce_scatter(dtype, op, k, off):
    c = get_comm(k, 2)
    for m in (1, 777, 4099):
        xs = data(m + 11 * k + off, k, k * m, dtype)
        s = offset_views(xs, off)
        d = [torch.empty(m + off, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
        c.reduce_scatter(s, d, op=op, algo="ring", proto="direct")
        finish(c)
        want = oracle.reduce_scatter(xs, dtype, op, 2, chunk(dtype, 1))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"m={m} rank {r}")
    # in place: recvbuf r is block r of sendbuf r
    m = 1001
    xs = data(5, k, k * m, dtype)
    s = [to_dev(x) for x in xs]
    c.reduce_scatter(s, [t[r * m:(r + 1) * m] for r, t in enumerate(s)], op=op, algo="ring",
                     proto="direct")
    finish(c)
    want = oracle.reduce_scatter(xs, dtype, op, 2, chunk(dtype, 1))
    for r in range(k):
        assert_same(to_np(s[r][r * m:(r + 1) * m], dtype), want[r], f"in place rank {r}")


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
@pytest.mark.parametrize("k", [2, 7, 16])
@pytest.mark.parametrize("off", [0, 1])
def test_all_gather(dtype, k, off):
    c = get_comm(k, 3)
    for m in (1, 999, 5000):
        xs = data(m + 5 * k + off, k, m, dtype)
        s = offset_views(xs, off)
        d = [torch.empty(k * m + off, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto="direct")
        finish(c)
        want = np.concatenate(xs)
        for r in range(k):
            assert_same(to_np(d[r], dtype), want, f"m={m} rank {r}")
    # in place: sendbuf r is block r of recvbuf r
    m = 640
    xs = data(3, k, m, dtype)
    d = [torch.empty(k * m, dtype=torch.float32 if dtype == "fp32" else torch.bfloat16,
                     device="cuda") for _ in range(k)]
    for r in range(k):
        d[r][r * m:(r + 1) * m].copy_(to_dev(xs[r]))
    c.all_gather([d[r][r * m:(r + 1) * m] for r in range(k)], d, algo="ring", proto="direct")
    finish(c)
    for r in range(k):
        assert_same(to_np(d[r], dtype), np.concatenate(xs), f"in place rank {r}")


@pytest.mark.parametrize("k,root", [(2, 1), (5, 0), (16, 9)])
def test_broadcast(k, root):
    c = get_comm(k, 2)
    for n in (1, 3000, 40001):
        xs = data(n + root, k, n, "fp16")
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        d[root] = s[root]                                 # the root in place
        c.broadcast(s, d, root=root, algo="ring", proto="direct")
        finish(c)
        for r in range(k):
            assert_same(to_np(d[r], "fp16"), xs[root], f"n={n} rank {r}")


@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("int32", "max"), ("bf16", "sum")])
@pytest.mark.parametrize("k,root", [(2, 0), (5, 3), (16, 15)])
def test_reduce(dtype, op, k, root):
    c = get_comm(k, 1)
    for n in (1, 2049, 30011):
        xs = data(n + 7 * root, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(s[0]) if r == root else None for r in range(k)]
        c.reduce(s, d, op=op, root=root, algo="ring", proto="direct")
        finish(c)
        want = oracle.reduce(xs, dtype, op, root, 1, chunk(dtype, 1))
        assert_same(to_np(d[root], dtype), want, f"n={n}")


def test_tree_is_unsupported_and_auto_takes_ring():
    k = 4
    c = get_comm(k, 2)
    s = [torch.ones(1000, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    with pytest.raises(VcommError) as e:
        c.all_reduce(s, d, algo="tree", proto="direct")
    assert e.value.name == "vUnsupported"
    c.all_reduce(s, d, algo="auto", proto="direct")
    finish(c)
    assert c.last_plan()["algo"] == "ring" and c.last_plan()["proto"] == "direct"
    assert float(d[2][5]) == 4.0


def test_group_of_several_direct_calls():
    k, n = 4, 5000
    c = get_comm(k, 4)
    xs = [data(60 + i, k, n, "fp32") for i in range(3)]
    ss = [[to_dev(x) for x in x3] for x3 in xs]
    dd = [[torch.empty_like(t) for t in s] for s in ss]
    with group():
        for s, d in zip(ss, dd):
            c.all_reduce(s, d, op="sum", algo="ring", proto="direct")
    finish(c)
    plans = c.group_plans()
    assert all(p["proto"] == "direct" for p in plans)
    for x3, d, p in zip(xs, dd, plans):
        want = oracle.all_reduce(x3, "fp32", "sum", p["nchannels"], chunk("fp32", p["chunkSteps"]))
        for r in range(k):
            assert_same(to_np(d[r], "fp32"), want[r], f"rank {r}")


def test_headline_size_sampled():
    """8 vranks x 256 MiB fp32, 37 channels: sampled elements against the
    oracle's one-element queries, and every element equal to a Simple call."""
    k, n, C = 8, (256 << 20) // 4, 37
    g = torch.Generator(device="cuda").manual_seed(5)
    s = [torch.randn(n, device="cuda", generator=g) for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c = Comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    c.all_reduce(s, d, algo="ring", proto="direct")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4000), [0, n - 1]]))
    t = torch.from_numpy(idx).cuda()
    full = [x.cpu().numpy() for x in s]
    want = oracle.all_reduce_points(full, idx, "fp32", "sum", C, chunk_for("simple", "fp32", None, 1))
    del full
    for r in (0, 3, 7):
        assert_same(d[r][t].cpu().numpy(), want, f"rank {r}")
    ref = [torch.empty_like(x) for x in s[:2]]
    c.all_reduce(s, [ref[0], ref[1]] + d[2:], algo="ring", proto="simple")
    torch.cuda.synchronize()
    assert torch.equal(ref[0].view(torch.int32), d[0].view(torch.int32))
    assert torch.equal(ref[1].view(torch.int32), d[1].view(torch.int32))
    c.destroy()


def test_mixed_group_in_one_launch():
    """40 direct calls of every collective, dtype, op and size (down to a
    single element, some on unaligned views) in one group: each result equals
    the oracle's for its own plan."""
    k = 6
    c = get_comm(k, 4)
    rng = np.random.default_rng(11)
    colls = ("allreduce", "reducescatter", "allgather", "broadcast", "reduce")
    calls = []
    with group():
        for i in range(40):
            coll = colls[i % 5]
            dtype = ("fp32", "bf16", "fp16", "int32")[int(rng.integers(4))]
            op = ("sum", "max")[int(rng.integers(2))]
            n = int(rng.choice([1, 3, 17, 1000, 4099, 65537]))
            off = int(rng.integers(2)) if n > 3 else 0
            root = int(rng.integers(k))
            m = k * n if coll == "reducescatter" else n
            xs = data(1000 + i, k, m, dtype)
            s = offset_views(xs, off)
            outn = n if coll != "allgather" else k * n
            d = [torch.empty(outn + off, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
            if coll == "allreduce":
                c.all_reduce(s, d, op=op, algo="ring", proto="direct")
            elif coll == "reducescatter":
                c.reduce_scatter(s, d, op=op, algo="ring", proto="direct")
            elif coll == "allgather":
                c.all_gather(s, d, algo="ring", proto="direct")
            elif coll == "broadcast":
                c.broadcast(s, d, root=root, algo="ring", proto="direct")
            else:
                d = [t if r == root else None for r, t in enumerate(d)]
                c.reduce(s, d, op=op, root=root, algo="ring", proto="direct")
            calls.append((coll, dtype, op, root, xs, s, d))
    finish(c)
    plans = c.group_plans()
    assert len(plans) == 40 and all(p["proto"] == "direct" for p in plans)
    for (coll, dtype, op, root, xs, s, d), p in zip(calls, plans):
        C, ch = p["nchannels"], chunk_for("direct", dtype, SMALL_SLOTS, p["chunkSteps"])
        if coll == "allreduce":
            want = oracle.all_reduce(xs, dtype, op, C, ch)
        elif coll == "reducescatter":
            want = oracle.reduce_scatter(xs, dtype, op, C, ch)
        elif coll == "allgather":
            want = [np.concatenate(xs)] * k
        elif coll == "broadcast":
            want = [xs[root]] * k
        else:
            assert_same(to_np(d[root], dtype), oracle.reduce(xs, dtype, op, root, C, ch), coll)
            continue
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"{coll} {dtype} {op} rank {r}")
