"""Failure detection without a GPU fault: a vrank that never takes part makes
its peers' bounded flag waits run out; the host reads vTimeout (or vAborted
after vcommAbort), the kernel returns, and the device stays usable."""
import time

import pytest

from paper_2507_04786_b300 import Comm, VcommError

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
@pytest.mark.parametrize("algo", ["ring", "tree"])
def test_lost_vrank_times_out(proto, algo):
    k = 4
    c = Comm(k, 2, slot_bytes={"simple": 8192, "ll": 2048, "ll128": 2560}, timeout_sec=0.2)
    s = [torch.ones(100000, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c.all_reduce(s, d, algo=algo, proto=proto)          # a healthy call first
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    c.debug_skip_rank(2)
    t0 = time.time()
    c.all_reduce(s, d, algo=algo, proto=proto)
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert c.async_error() == "vTimeout"
    with pytest.raises(VcommError) as e:                # a failed communicator stays failed
        c.all_reduce(s, d, algo=algo, proto=proto)
    assert e.value.name == "vTimeout"
    c.destroy()
    # the device is still usable: a fresh communicator works
    c2 = Comm(k, 2)
    c2.all_reduce(s, d, algo="ring", proto=proto)
    torch.cuda.synchronize()
    assert c2.async_error() == "vSuccess"
    assert float(d[0][0]) == float(k)
    c2.destroy()


def test_abort_ends_a_blocked_call():
    """ncclCommAbort (Sec. II-A-1): the abort word ends in-flight waits long
    before their deadline."""
    k = 4
    c = Comm(k, 1, timeout_sec=30.0)
    s = [torch.ones(1 << 20, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c.debug_skip_rank(0)
    t0 = time.time()
    c.all_reduce(s, d, algo="ring", proto="simple")
    time.sleep(0.2)
    c.abort()                                            # raises the abort word, waits, frees
    assert time.time() - t0 < 10.0
    x = torch.ones(10, device="cuda")
    assert float((x * 2).sum()) == 20.0


# ---------------------------------------------------------------- recovery

@pytest.mark.parametrize("proto,algo", [("simple", "ring"), ("ll", "tree"), ("ll128", "ring"),
                                        ("cluster", "ring"), ("cluster", "tree")])
def test_reset_after_a_timeout_reuses_the_comm(proto, algo):
    """A lost vrank times out; vcommReset re-zeroes the FIFOs and clears the
    error; the same communicator then runs exact collectives again."""
    import numpy as np

    import oracle
    from gpu_util import assert_same, chunk_for, to_dev, to_np
    from paper_2507_04786_b300 import inputs
    k, n = 4, 100003
    slots = {"simple": 8192, "ll": 2048, "ll128": 2560}
    c = Comm(k, 2, slot_bytes=slots, timeout_sec=0.2)
    xs = inputs.workload(5, k, n, "fp32", "normal")
    s = [to_dev(x) for x in xs]
    d = [torch.empty_like(t) for t in s]
    c.set_plan(nchannels=2, chunk_steps=1)
    c.debug_skip_rank(1)
    c.all_reduce(s, d, algo=algo, proto=proto)
    torch.cuda.synchronize()
    assert c.async_error() == "vTimeout"
    c.reset()
    assert c.async_error() == "vSuccess"
    for rep in range(2):                      # twice: the counters restart cleanly
        c.all_reduce(s, d, algo=algo, proto=proto)
        torch.cuda.synchronize()
        assert c.async_error() == "vSuccess"
        p = c.last_plan()
        want = oracle.all_reduce(xs, "fp32", "sum", p["nchannels"],
                                 chunk_for(p["proto"], "fp32", slots, p["chunkSteps"]), p["algo"])
        for r in range(k):
            assert_same(to_np(d[r], "fp32"), want[r], f"rep {rep} rank {r}")
    c.destroy()


def test_abort_pending_then_reset():
    """Abort a blocked call without destroying the communicator: the kernel
    returns vAborted long before its deadline; after a reset the
    communicator works."""
    k = 4
    c = Comm(k, 1, timeout_sec=30.0)
    s = [torch.ones(1 << 20, device="cuda") for _ in range(k)]
    d = [torch.empty_like(t) for t in s]
    c.debug_skip_rank(0)
    t0 = time.time()
    c.all_reduce(s, d, algo="ring", proto="simple")
    time.sleep(0.2)
    c.abort_pending()
    assert time.time() - t0 < 10.0
    assert c.async_error() == "vAborted"
    with pytest.raises(VcommError):
        c.all_reduce(s, d, algo="ring", proto="simple")
    c.reset()
    c.all_reduce(s, d, algo="ring", proto="simple")
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    assert float(d[2][12345]) == float(k)
    c.destroy()
