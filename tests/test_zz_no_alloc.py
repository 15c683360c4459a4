"""The allocation-free AllReduce (vAllReduceNoAlloc) gives the same bits as the
ordinary vAllReduce with the same plan.

vAllReduceNoAlloc serves callers that cannot allocate device memory when they
need the collective (a fixed memory budget owned by another allocator, or a
latency-critical path where cudaMalloc / cudaFree could block or synchronise
the device): its FIFOs live in a fixed device array inside the library.  The
check runs two calls in a row, because every call reuses that array and must
clear what the previous call left in it.  This file is collected last so that
a failure here stops a `-x` run only after every other test has run; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2507_04786_b300 import Comm, inputs, load_library
from paper_2507_04786_b300.binding import DTYPE_CODES, OP_CODES, RESULTS

from gpu_util import assert_same, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ptrs(ts):
    a = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        a[i] = t.data_ptr()
    return a


@pytest.mark.parametrize("dtype,op,dist", [("fp32", "sum", "normal"), ("bf16", "max", "normal")])
def test_no_alloc_allreduce_matches_vallreduce(dtype, op, dist):
    assert torch.cuda.is_available()
    L = load_library()
    k, C, n = 8, 4, 1_000_003
    xs = inputs.workload(91, k, n, dtype, dist)
    sends = [to_dev(x) for x in xs]
    # the existing entry point with the same plan: ring, Simple, C channels,
    # 64 KiB Simple slots, one slot per chunk
    comm = Comm(k, C, slot_bytes={"simple": 64 * 1024})
    comm.set_plan(nchannels=C, chunk_steps=1)
    ref = [torch.empty_like(s) for s in sends]
    comm.all_reduce(sends, ref, op=op, algo="ring", proto="simple")
    torch.cuda.synchronize()
    assert comm.async_error() == "vSuccess"
    comm.destroy()
    want = [to_np(t, dtype) for t in ref]

    status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        outs = [torch.full_like(s, 7) for s in sends]
        rc = L.vAllReduceNoAlloc(_ptrs(sends), _ptrs(outs), n, DTYPE_CODES[dtype], OP_CODES[op],
                                 k, C, ctypes.c_void_p(status.data_ptr()), stream)
        assert RESULTS[rc] == "vSuccess"
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, 0, 0, 0], f"call {call}"
        for r in range(k):
            assert_same(to_np(outs[r], dtype), want[r], f"call {call} rank {r}")


def test_no_alloc_rejects_too_many_connections():
    L = load_library()
    a = [torch.zeros(16, device="cuda") for _ in range(8)]
    rc = L.vAllReduceNoAlloc(_ptrs(a), _ptrs(a), 16, DTYPE_CODES["fp32"], OP_CODES["sum"],
                             8, 5, None, torch.cuda.current_stream().cuda_stream)
    assert RESULTS[rc] == "vInvalidArgument"      # 8 x 5 = 40 > 32 connections
    torch.cuda.synchronize()
