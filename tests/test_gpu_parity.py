"""GPU parity: every collective through the C ABI against the CPU oracle.

Bit-exact comparisons on the same seeded inputs, for every protocol, dtype,
op, channel count and a range of ragged sizes; small FIFO slots make modest
sizes span many loops, chunks and FIFO steps.  The full-size headline case is
checked on sampled elements the oracle computes one at a time.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs, workloads
from paper_2507_04786_b300.binding import debug_decode, debug_encode

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "fp16": ("uniform", {}),
        "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}

_comms = {}


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    assert torch.cuda.is_available()
    yield
    for c in _comms.values():
        c.destroy()
    _comms.clear()


def get_comm(k, C, slots=SMALL_SLOTS):
    key = (k, C, None if slots is None else tuple(sorted(slots.items())))
    if key not in _comms:
        _comms[key] = Comm(k, C, slot_bytes=slots, timeout_sec=10.0)
    return _comms[key]


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


# ---------------------------------------------------------------- the exact case

def test_exact_case_4vr_1Mi():
    """4 vranks, fp32 integers in [-1000, 1000] (exact sums), Simple, 1
    channel, default slots: bit-exact against the oracle and the plain sum."""
    w = workloads.EXACT
    k, n = w["nranks"], w["count"]
    xs = inputs.workload(w["seed"], k, n, "fp32", "int", lo=-1000, hi=1000)
    c = get_comm(k, 1, slots=None)
    c.set_plan(nchannels=1, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, op="sum", algo="ring", proto="simple")
    finish(c)
    want = oracle.all_reduce(xs, "fp32", "sum", 1, chunk_for("simple", "fp32"))
    plain = np.sum(np.stack(xs).astype(np.float64), axis=0).astype(np.float32)
    for r in range(k):
        got = to_np(d[r], "fp32")
        assert_same(got, want[r], f"rank {r}")
        assert_same(got, plain, f"rank {r} vs plain sum")


# ---------------------------------------------------------------- ring AllReduce

@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("dtype", ["fp32", "bf16", "fp16", "int32"])
@pytest.mark.parametrize("op", ["sum", "max"])
@pytest.mark.parametrize("k,C", [(2, 1), (3, 3), (8, 2)])
@pytest.mark.parametrize("n", [5, 20011])
def test_ring_allreduce(proto, dtype, op, k, C, n):
    xs = data(1000 + n + k, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, op=op, algo="ring", proto=proto)
    finish(c)
    want = oracle.all_reduce(xs, dtype, op, C, chunk_for(proto, dtype, SMALL_SLOTS))
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r}")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("chunk_steps", [2, 3])
def test_ring_allreduce_multi_slot_chunks(proto, chunk_steps):
    """chunkCount spanning several FIFO slots (chunkSteps > 1)."""
    k, C, n, dtype = 4, 2, 50021, "bf16"
    xs = data(77, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=chunk_steps)
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, op="sum", algo="ring", proto=proto)
    finish(c)
    want = oracle.all_reduce(xs, dtype, "sum", C, chunk_for(proto, dtype, SMALL_SLOTS, chunk_steps))
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r}")


# ---------------------------------------------------------------- tree AllReduce

@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max"),
                                      ("int32", "sum"), ("fp16", "sum")])
@pytest.mark.parametrize("k,C", [(2, 1), (3, 1), (5, 2), (8, 1), (16, 2)])
def test_tree_allreduce(proto, dtype, op, k, C):
    n = 30011
    xs = data(2000 + k, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, op=op, algo="tree", proto=proto)
    finish(c)
    want = oracle.all_reduce(xs, dtype, op, C, chunk_for(proto, dtype, SMALL_SLOTS), "tree")
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r}")


# ---------------------------------------------------------------- RS / AG / Bcast / Reduce

@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("dtype,op", [("fp16", "sum"), ("int32", "max"), ("fp32", "sum"),
                                      ("bf16", "max")])
@pytest.mark.parametrize("k,C", [(2, 1), (8, 2), (16, 1)])
@pytest.mark.parametrize("n", [16, 9001])
def test_reduce_scatter(proto, dtype, op, k, C, n):
    xs = data(3000 + n, k, k * n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.empty(n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
    c.reduce_scatter(s, d, op=op, algo="ring", proto=proto)
    finish(c)
    want = oracle.reduce_scatter(xs, dtype, op, C, chunk_for(proto, dtype, SMALL_SLOTS))
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r}")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("dtype", ["fp16", "int32"])
@pytest.mark.parametrize("k,C", [(2, 1), (8, 3), (16, 1)])
@pytest.mark.parametrize("n", [8, 7001])
def test_all_gather(proto, dtype, k, C, n):
    xs = data(4000 + n, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    s = [to_dev(x) for x in xs]
    d = [torch.empty(k * n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
    c.all_gather(s, d, algo="ring", proto=proto)
    finish(c)
    want = oracle.all_gather(xs, C, chunk_for(proto, dtype, SMALL_SLOTS, byte_units=True))
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r}")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("k,C", [(2, 1), (8, 2), (16, 1)])
def test_broadcast_all_roots(proto, k, C):
    n, dtype = 12345, "fp16"
    xs = data(5000 + k, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    for root in sorted({0, 1, k - 1}):
        s = [to_dev(x) if r == root else None for r, x in enumerate(xs)]
        d = [torch.empty(n, dtype=torch.float16, device="cuda") for _ in range(k)]
        c.broadcast(s, d, root=root, algo="ring", proto=proto)
        finish(c)
        want = oracle.broadcast(xs, root, C, chunk_for(proto, dtype, SMALL_SLOTS, byte_units=True))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"root {root} rank {r}")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("dtype,op", [("fp16", "sum"), ("int32", "max"), ("bf16", "sum")])
@pytest.mark.parametrize("k,C", [(2, 1), (8, 2), (16, 1)])
def test_reduce_all_roots(proto, dtype, op, k, C):
    n = 10007
    xs = data(6000 + k, k, n, dtype)
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    for root in sorted({0, 1, k - 1}):
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(s[0]) if r == root else None for r in range(k)]
        c.reduce(s, d, op=op, root=root, algo="ring", proto=proto)
        finish(c)
        want = oracle.reduce(xs, dtype, op, root, C, chunk_for(proto, dtype, SMALL_SLOTS))
        assert_same(to_np(d[root], dtype), want, f"root {root}")


# ---------------------------------------------------------------- in place

@pytest.mark.parametrize("proto", ["simple", "ll128", "ll"])
def test_in_place_forms(proto):
    """Sec. II-A-2 / V-E: in-place AllReduce, AllGather (send = own block of
    recv), ReduceScatter (recv = own block of send), Broadcast and Reduce
    (ncclBcast form) equal the out-of-place results."""
    k, C, n, dtype = 4, 2, 4099, "fp32"
    c = get_comm(k, C)
    c.set_plan(nchannels=C, chunk_steps=1)
    ch = chunk_for(proto, dtype, SMALL_SLOTS)
    chb = chunk_for(proto, dtype, SMALL_SLOTS, byte_units=True)
    xs = data(7001, k, n, dtype)
    # AllReduce
    buf = [to_dev(x) for x in xs]
    c.all_reduce(buf, buf, algo="ring", proto=proto)
    finish(c)
    want = oracle.all_reduce(xs, dtype, "sum", C, ch)
    for r in range(k):
        assert_same(to_np(buf[r], dtype), want[r], f"AR rank {r}")
    buf = [to_dev(x) for x in xs]
    c.all_reduce(buf, buf, algo="tree", proto=proto)
    finish(c)
    want = oracle.all_reduce(xs, dtype, "sum", C, ch, "tree")
    for r in range(k):
        assert_same(to_np(buf[r], dtype), want[r], f"tree AR rank {r}")
    # AllGather
    big = [torch.zeros(k * n, dtype=torch.float32, device="cuda") for _ in range(k)]
    for r in range(k):
        big[r][r * n:(r + 1) * n] = to_dev(xs[r])
    c.all_gather([big[r][r * n:(r + 1) * n] for r in range(k)], big, algo="ring", proto=proto)
    finish(c)
    want = oracle.all_gather(xs, C, chb)
    for r in range(k):
        assert_same(to_np(big[r], dtype), want[r], f"AG rank {r}")
    # ReduceScatter
    xrs = data(7002, k, k * n, dtype)
    big = [to_dev(x) for x in xrs]
    c.reduce_scatter(big, [big[r][r * n:(r + 1) * n] for r in range(k)], algo="ring", proto=proto)
    finish(c)
    want = oracle.reduce_scatter(xrs, dtype, "sum", C, ch)
    for r in range(k):
        assert_same(to_np(big[r][r * n:(r + 1) * n], dtype), want[r], f"RS rank {r}")
    # Broadcast, in place at the root
    buf = [to_dev(x) for x in xs]
    c.broadcast([buf[r] if r == 1 else None for r in range(k)], buf, root=1, algo="ring",
                proto=proto)
    finish(c)
    for r in range(k):
        assert_same(to_np(buf[r], dtype), xs[1], f"bcast rank {r}")
    # Reduce, in place at the root
    buf = [to_dev(x) for x in xs]
    c.reduce(buf, [buf[r] if r == 2 else None for r in range(k)], root=2, algo="ring", proto=proto)
    finish(c)
    assert_same(to_np(buf[2], dtype), oracle.reduce(xs, dtype, "sum", 2, C, ch), "reduce root")


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
def test_unaligned_blocks(proto):
    """ReduceScatter / AllGather blocks that are not 16-byte aligned take the
    element-wise paths."""
    k, C = 3, 2
    for dtype, n in (("fp16", 13), ("fp32", 3), ("bf16", 1001)):
        c = get_comm(k, C)
        c.set_plan(nchannels=C, chunk_steps=1)
        xs = data(8000 + n, k, k * n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.reduce_scatter(s, d, algo="ring", proto=proto)
        finish(c)
        want = oracle.reduce_scatter(xs, dtype, "sum", C, chunk_for(proto, dtype, SMALL_SLOTS))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"RS {dtype} rank {r}")
        ys = data(8100 + n, k, n, dtype)
        s = [to_dev(y) for y in ys]
        d = [torch.empty(k * n, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto=proto)
        finish(c)
        want = oracle.all_gather(ys, C, chunk_for(proto, dtype, SMALL_SLOTS, byte_units=True))
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"AG {dtype} rank {r}")


def test_single_rank_and_empty():
    c = get_comm(1, 2)
    c.set_plan(nchannels=2, chunk_steps=1)
    x = data(9, 1, 1000, "bf16")
    s = [to_dev(x[0])]
    for fn in ("all_reduce", "broadcast", "reduce"):
        d = [torch.empty_like(s[0])]
        getattr(c, fn)(s, d)
        finish(c)
        assert_same(to_np(d[0], "bf16"), x[0], fn)
    d = [torch.empty_like(s[0])]
    c.all_gather(s, d)
    c.reduce_scatter(s, d)
    finish(c)
    assert_same(to_np(d[0], "bf16"), x[0], "rs/ag")
    # count 0 is a no-op
    c2 = get_comm(4, 1)
    e = [torch.empty(0, device="cuda") for _ in range(4)]
    c2.all_reduce(e, e)
    finish(c2)


def test_max_ranks_64():
    k, n = 64, 3001
    xs = data(64, k, n, "fp32")
    c = get_comm(k, 1)
    c.set_plan(nchannels=1, chunk_steps=1)
    for proto in ("simple", "ll128", "ll"):
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, algo="ring", proto=proto)
        finish(c)
        want = oracle.all_reduce(xs, "fp32", "sum", 1, chunk_for(proto, "fp32", SMALL_SLOTS))
        for r in (0, 17, 63):
            assert_same(to_np(d[r], "fp32"), want[r], f"{proto} rank {r}")


def test_argument_errors():
    from paper_2507_04786_b300 import VcommError
    c = get_comm(4, 1)
    a = [torch.zeros(100, device="cuda") for _ in range(4)]
    b = [torch.zeros(100, device="cuda") for _ in range(4)]
    with pytest.raises(VcommError) as e:
        c.all_gather(a, b, algo="tree")              # tree is AllReduce-only
    assert e.value.name == "vUnsupported"
    with pytest.raises(VcommError) as e:
        c.all_reduce(a, [b[0], b[0], b[1], b[2]])     # two ranks share an output
    assert e.value.name == "vInvalidArgument"
    with pytest.raises(VcommError) as e:
        c.all_reduce([a[0][1:], a[1][1:], a[2][1:], a[3][1:]], [a[0][:99], b[1][:99], b[2][:99],
                                                                 b[3][:99]])  # partial overlap
    assert e.value.name == "vInvalidArgument"
    with pytest.raises(VcommError) as e:
        c.broadcast(a, b, root=4)
    assert e.value.name == "vInvalidArgument"
    finish(c)


# ---------------------------------------------------------------- plan / tuner

def test_auto_plan_is_reported_and_exact():
    k, n, dtype = 8, 70001, "bf16"
    xs = data(31, k, n, dtype)
    c = get_comm(k, 4)
    c.clear_plan()
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, algo="auto", proto="auto")
    finish(c)
    p = c.last_plan()
    want = oracle.all_reduce(xs, dtype, "sum", p["nchannels"],
                             chunk_for(p["proto"], dtype, SMALL_SLOTS, p["chunkSteps"]), p["algo"])
    for r in range(k):
        assert_same(to_np(d[r], dtype), want[r], f"rank {r} plan {p}")


# ---------------------------------------------------------------- protocol encodings

@pytest.mark.parametrize("proto", ["ll", "ll128"])
@pytest.mark.parametrize("nbytes", [1, 7, 8, 120, 121, 4000, 576000])
def test_line_encoding_matches_oracle(proto, nbytes):
    """Sec. III-B / III-C: the device encoder writes exactly the oracle's lines."""
    g = np.random.default_rng(nbytes)
    data_ = g.integers(0, 256, nbytes, dtype=np.uint8)
    src = torch.from_numpy(data_).cuda()
    flag = 0x1234567 if proto == "ll" else 0x0123456789AB
    if proto == "ll":
        want = oracle.ll_encode(data_, flag)
        nl = ((nbytes + 7) // 8) * 2
        lines = torch.zeros(nl, dtype=torch.int64, device="cuda")
    else:
        want = oracle.ll128_encode(data_, flag)
        lines = torch.zeros(want.size, dtype=torch.int64, device="cuda")
    debug_encode(proto, src, nbytes, flag, lines)
    torch.cuda.synchronize()
    got = lines.cpu().numpy().view(np.uint64)[:want.size]
    assert np.array_equal(got, want)
    dst = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    assert debug_decode(proto, lines, nbytes, flag, dst) == "vSuccess"
    assert np.array_equal(dst.cpu().numpy(), data_)


@pytest.mark.parametrize("proto", ["ll", "ll128"])
def test_stale_flag_wait_times_out(proto):
    """A reader waiting for a flag nobody writes gives up at its deadline and
    reports vTimeout; the context stays usable."""
    nbytes = 240
    lines = torch.zeros(64, dtype=torch.int64, device="cuda")
    debug_encode(proto, torch.zeros(nbytes, dtype=torch.uint8, device="cuda"), nbytes, 5, lines)
    dst = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    assert debug_decode(proto, lines, nbytes, 6, dst, timeout_sec=0.2) == "vTimeout"
    assert debug_decode(proto, lines, nbytes, 5, dst, timeout_sec=0.2) == "vSuccess"
    x = torch.ones(10, device="cuda")
    assert float((x + 1).sum()) == 20.0


# ---------------------------------------------------------------- full size, sampled

@pytest.mark.parametrize("proto", workloads.HEADLINE["protos"])
def test_headline_full_size_sampled(proto):
    """The benchmark's launch configuration at its full size (8 vranks x
    256 MiB fp32): every rank bit-identical, and sampled elements equal the
    oracle's one-element replay."""
    w = workloads.HEADLINE
    k, C = w["nranks"], w["nchannels"]
    n = w["bytes_per_rank"] // 4
    xs = inputs.workload(w["seed"], k, n, "fp32", w["dist"])
    c = get_comm(k, C, slots=None)
    c.set_plan(nchannels=C, chunk_steps=w["chunk_steps"])
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, op="sum", algo="ring", proto=proto)
    finish(c)
    for r in range(1, k):
        assert torch.equal(d[r].view(torch.int32), d[0].view(torch.int32)), f"rank {r} differs"
    g = np.random.default_rng(5)
    idx = np.unique(np.concatenate([g.integers(0, n, 20000), [0, 1, n - 1, n // 2, n // C]]))
    chunk = chunk_for(proto, "fp32", None, w["chunk_steps"])
    want = oracle.all_reduce_points(xs, idx, "fp32", "sum", C, chunk, "ring")
    got = d[3][torch.from_numpy(idx).cuda()].cpu().numpy()
    assert_same(got, want, "sampled")
    c.destroy()
    _comms.pop((k, C, None))
