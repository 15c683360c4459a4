"""GPU parity of point-to-point transfers (vSend / vRecv in groups) and
all-to-all against the oracle's plain definitions, byte-exact.

Covered: all-to-all on 1..16 vranks, every dtype, empty, odd and unaligned
blocks, inside and outside a group, captured in a CUDA graph; grouped
send / receive patterns (ring shift, random permutation, many-to-one,
one-to-many, several transfers per pair in issue order, self-copy) mixed with
a collective in the same group; and the refusals: a call outside a group, an
unmatched or mismatched transfer (the whole group is refused and nothing
runs).
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, VcommError, group, inputs
from paper_2507_04786_b300.binding import group_end, group_start

from gpu_util import assert_same, to_dev, to_np

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


def get_comm(k):
    if k not in _comms:
        _comms[k] = Comm(k, 2, timeout_sec=10.0)
    return _comms[k]


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


def dev_views(xs, off):
    out = []
    for x in xs:
        t = to_dev(np.concatenate([x[:1].repeat(off), x]) if off else x)
        out.append(t[off:])
    return out


@pytest.mark.parametrize("k", [1, 2, 5, 8, 16])
@pytest.mark.parametrize("dtype", ["fp32", "bf16", "int32", "fp16"])
@pytest.mark.parametrize("n", [0, 1, 7, 4096, 30001])
def test_all_to_all(k, dtype, n):
    c = get_comm(k)
    xs = data(n + 3 * k, k, k * n, dtype)
    off = 1 if n == 7 else 0                     # odd element offsets take the byte path
    s = dev_views(xs, off)
    d = [torch.full((k * n + off,), 0, dtype=s[0].dtype, device="cuda")[off:] for _ in range(k)]
    c.all_to_all(s, d, count=n)
    finish(c)
    if n == 0:
        return
    want = oracle.all_to_all(xs)
    for j in range(k):
        assert_same(to_np(d[j], dtype), want[j], f"rank {j}")


def test_all_to_all_in_a_group_and_a_graph():
    k, n = 8, 5000
    c = get_comm(k)
    xs = data(1, k, k * n, "fp32")
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    with group():
        c.all_to_all(s, d)
    finish(c)
    want = oracle.all_to_all(xs)
    for j in range(k):
        assert_same(to_np(d[j], "fp32"), want[j], f"group rank {j}")
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        c.all_to_all(s, d, stream=stream)
    ys = data(2, k, k * n, "fp32")
    for t, y in zip(s, ys):
        t.copy_(to_dev(y))
    torch.cuda.synchronize()
    g.replay()
    finish(c)
    want = oracle.all_to_all(ys)
    for j in range(k):
        assert_same(to_np(d[j], "fp32"), want[j], f"graph rank {j}")


def run_pattern(c, pairs, n, dtype, seed):
    """Issue sends and receives for `pairs` (src, dst) in one group; return
    the sent arrays, the receive tensors and the oracle's matched results."""
    rng = np.random.default_rng(seed)
    sends, recvs, outs = [], [], []
    group_start()
    try:
        for i, (a, b) in enumerate(pairs):
            m = int(n + rng.integers(0, 3))
            x = data(seed * 1000 + i, 1, m, dtype)[0]
            t = to_dev(x)
            sends.append((a, b, x))
            c.send(a, b, t)
            r = torch.empty_like(t)
            recvs.append((b, a, m))
            outs.append((r, t))
            c.recv(b, a, r)
    finally:
        group_end()
    finish(c)
    want = oracle.p2p_match(sends, recvs)
    return outs, want


@pytest.mark.parametrize("pattern", ["ring", "perm", "to_one", "from_one", "repeat", "self"])
@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_grouped_send_recv(pattern, dtype):
    k = 6
    c = get_comm(k)
    rng = np.random.default_rng(3)
    if pattern == "ring":
        pairs = [(r, (r + 1) % k) for r in range(k)]
    elif pattern == "perm":
        p = rng.permutation(k)
        pairs = [(r, int(p[r])) for r in range(k)]
    elif pattern == "to_one":
        pairs = [(r, 2) for r in range(k) if r != 2]
    elif pattern == "from_one":
        pairs = [(4, r) for r in range(k) if r != 4]
    elif pattern == "repeat":                   # several transfers per pair: issue order
        pairs = [(1, 3), (1, 3), (0, 5), (1, 3), (5, 0)]
    else:
        pairs = [(r, r) for r in range(k)]
    outs, want = run_pattern(c, pairs, 4099, dtype, seed=len(pattern))
    for (r, _), w in zip(outs, want):
        assert_same(to_np(r, dtype), w, pattern)


def test_p2p_and_a_collective_in_one_group():
    k, n = 4, 3000
    c = get_comm(k)
    xs = data(9, k, n, "fp32")
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    a = to_dev(data(10, 1, 777, "fp32")[0])
    b = torch.empty_like(a)
    with group():
        c.all_reduce(s, d, op="sum", algo="ring", proto="direct")
        c.send(0, 3, a)
        c.recv(3, 0, b)
    finish(c)
    assert torch.equal(a, b)
    p = c.group_plans()[0]
    want = oracle.all_reduce(xs, "fp32", "sum", p["nchannels"],
                             oracle.chunk_units("simple", 4, p["chunkSteps"]))
    for r in range(k):
        assert_same(to_np(d[r], "fp32"), want[r], f"rank {r}")


def test_refusals():
    k = 3
    c = get_comm(k)
    t = torch.ones(100, device="cuda")
    r = torch.zeros(100, device="cuda")
    with pytest.raises(VcommError) as e:           # outside a group
        c.send(0, 1, t)
    assert e.value.name == "vInvalidArgument"
    with pytest.raises(VcommError) as e:           # a send without its receive
        with group():
            c.send(0, 1, t)
    assert e.value.name == "vInvalidArgument"
    with pytest.raises(VcommError) as e:           # counts disagree: nothing runs
        with group():
            c.send(0, 1, t)
            c.recv(1, 0, r, count=50)
    assert e.value.name == "vInvalidArgument"
    torch.cuda.synchronize()
    assert float(r.sum()) == 0.0
    with pytest.raises(VcommError) as e:           # peer out of range
        with group():
            c.send(0, 3, t)
    assert e.value.name == "vInvalidArgument"
    assert c.async_error() == "vSuccess"
