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
