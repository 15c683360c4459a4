"""GPU parity of the copies staged through shared memory (kCopyStaged: one
thread per CTA moves 32 KiB tiles with bulk copies): AllGather, Broadcast,
all-to-all and grouped send / receive, byte-exact against the oracle.

The staged copies take 16-byte aligned tasks of whole 16-byte units from
VCOMM_STAGED_MIN_BYTES (per rank for AllGather and Broadcast, in total for
transfers), read when a communicator is created.  These tests create their
communicators with that threshold at 16 bytes, so modest sizes already span
many tiles, a ragged last tile, several tasks per CTA and, for 16 vranks'
all-to-all, several launches of 64 tasks; sizes that are not whole 16-byte
units take the register kernel and must give the same bytes.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, group, inputs

from gpu_util import assert_same, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_comms = {}


@pytest.fixture(scope="module", autouse=True)
def _cleanup():
    assert torch.cuda.is_available()
    yield
    for c in _comms.values():
        c.destroy()
    _comms.clear()


def make_comm(k, min_bytes):
    old = os.environ.get("VCOMM_STAGED_MIN_BYTES")
    os.environ["VCOMM_STAGED_MIN_BYTES"] = str(min_bytes)
    try:
        return Comm(k, 2, timeout_sec=10.0)
    finally:
        if old is None:
            del os.environ["VCOMM_STAGED_MIN_BYTES"]
        else:
            os.environ["VCOMM_STAGED_MIN_BYTES"] = old


def get_comm(k):
    if k not in _comms:
        _comms[k] = make_comm(k, 16)
    return _comms[k]


def data(seed, k, n, dtype="fp32"):
    return inputs.workload(seed, k, n, dtype, "normal")


def finish(c):
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"


@pytest.mark.parametrize("k", [2, 3, 8, 16, 64])
@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_all_gather(k, dtype):
    c = get_comm(k)
    sizes = (8, 1000, 16384, 100000, 1001) if k <= 16 else (8, 8192, 1001)
    for m in sizes:                      # 1001 x 4 or x 2 bytes: not whole units
        xs = data(m + k, k, m, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty(k * m, dtype=s[0].dtype, device="cuda") for _ in range(k)]
        c.all_gather(s, d, algo="ring", proto="direct")
        finish(c)
        want = np.concatenate(xs)
        for r in sorted({0, k // 2, k - 1}):
            assert_same(to_np(d[r], dtype), want, f"m={m} rank {r}")


@pytest.mark.parametrize("k", [2, 7, 16])
def test_all_gather_in_place(k):
    c = get_comm(k)
    m = 40000
    xs = data(3 * k, k, m)
    d = [torch.empty(k * m, device="cuda") for _ in range(k)]
    for r in range(k):
        d[r][r * m:(r + 1) * m].copy_(to_dev(xs[r]))
    c.all_gather([d[r][r * m:(r + 1) * m] for r in range(k)], d, algo="ring", proto="direct")
    finish(c)
    for r in range(k):
        assert_same(to_np(d[r], "fp32"), np.concatenate(xs), f"in place rank {r}")


@pytest.mark.parametrize("k,root", [(2, 1), (5, 0), (16, 9), (64, 63)])
def test_broadcast(k, root):
    c = get_comm(k)
    for n in (8, 3000, 40000, 300000, 40001):   # 40001 fp16: not whole units
        xs = data(n + root, k, n, "fp16")
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.broadcast(s, d, root=root, algo="ring", proto="direct")
        finish(c)
        for r in sorted({0, root, k - 1}):
            assert_same(to_np(d[r], "fp16"), xs[root], f"n={n} rank {r}")
        d[root] = s[root]                        # the root in place
        c.broadcast(s, d, root=root, algo="ring", proto="direct")
        finish(c)
        for r in sorted({0, root, k - 1}):
            assert_same(to_np(d[r], "fp16"), xs[root], f"in place n={n} rank {r}")


@pytest.mark.parametrize("k", [2, 8, 16])
@pytest.mark.parametrize("n", [4, 12288, 100000])
def test_all_to_all(k, n):
    c = get_comm(k)
    xs = data(n + 5 * k, k, k * n)
    s = [to_dev(x) for x in xs]
    d = [torch.zeros_like(t) for t in s]
    c.all_to_all(s, d, count=n)
    finish(c)
    want = oracle.all_to_all(xs)
    for j in range(k):
        assert_same(to_np(d[j], "fp32"), want[j], f"rank {j}")


def test_grouped_send_recv_and_self_copies():
    k = 6
    c = get_comm(k)
    pairs = [(1, 3), (1, 3), (0, 5), (2, 2), (1, 3), (5, 0), (4, 4)]
    sends, recvs, outs = [], [], []
    with group():
        for i, (a, b) in enumerate(pairs):
            x = data(100 + i, 1, 50000 + 4 * i)[0]
            t = to_dev(x)
            r = t if a == b and i == 6 else torch.empty_like(t)   # one self-copy in place
            sends.append((a, b, x))
            recvs.append((b, a, x.size))
            outs.append((r, t))
            c.send(a, b, t)
            c.recv(b, a, r)
    finish(c)
    want = oracle.p2p_match(sends, recvs)
    for (r, _), w in zip(outs, want):
        assert_same(to_np(r, "fp32"), w, "transfer")


def kernels_of(fn):
    prof = pytest.importorskip("torch.profiler")
    torch.cuda.synchronize()
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        fn()
        torch.cuda.synchronize()
    return [e.name for e in p.events()]


def test_threshold_picks_the_kernel():
    """The launch list shows the staged copy kernel at or above the
    threshold and the register kernel below it."""
    k = 4
    c = make_comm(k, 1 << 20)
    small = [torch.ones((1 << 20) // 4 - 4, device="cuda") for _ in range(k)]
    large = [torch.ones((1 << 20) // 4, device="cuda") for _ in range(k)]
    ds = [torch.empty(k * t.numel(), device="cuda") for t in small]
    dl = [torch.empty(k * t.numel(), device="cuda") for t in large]
    below = kernels_of(lambda: c.all_gather(small, ds, algo="ring", proto="direct"))
    above = kernels_of(lambda: c.all_gather(large, dl, algo="ring", proto="direct"))
    finish(c)
    c.destroy()
    assert float(dl[3][-1]) == 1.0 and float(ds[3][-1]) == 1.0
    if not above:
        pytest.skip("the profiler recorded no CUDA kernels")
    assert any("kCopyStaged" in x for x in above)
    assert not any("kCopyStaged" in x for x in below)
