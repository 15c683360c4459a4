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


def _reference(sends, k, C, dtype, op, inplace=()):
    """vAllReduce with the same plan: ring, Simple, C channels, 64 KiB Simple
    slots, one slot per chunk (in place for the ranks in `inplace`)."""
    comm = Comm(k, C, slot_bytes={"simple": 64 * 1024})
    comm.set_plan(nchannels=C, chunk_steps=1)
    srcs = [s.clone() for s in sends]
    outs = [srcs[r] if r in inplace else torch.empty_like(s) for r, s in enumerate(sends)]
    comm.all_reduce(srcs, outs, op=op, algo="ring", proto="simple")
    torch.cuda.synchronize()
    assert comm.async_error() == "vSuccess"
    comm.destroy()
    return [to_np(t, dtype) for t in outs]


# (vranks, channels, count, dtype, op, in-place ranks, pass a status buffer)
CASES = [
    (8, 4, 1_000_003, "fp32", "sum", (), True),
    (8, 4, 1_000_003, "bf16", "max", (), True),
    (1, 3, 70_001, "fp32", "sum", (), True),          # one vrank: a copy
    (1, 1, 4_097, "bf16", "sum", (0,), True),         # one vrank in place
    (5, 2, 333_337, "fp32", "sum", (0, 2, 4), True),  # in-place and out-of-place ranks mixed
    (3, 5, 262_147, "fp16", "sum", (), True),         # odd channel split, ragged count
    (4, 8, 500_001, "int32", "max", (1,), False),     # no status buffer
    (6, 5, 123_457, "bf16", "sum", (), False),
]


@pytest.mark.parametrize("k,C,n,dtype,op,inplace,with_status", CASES)
def test_no_alloc_allreduce_matches_vallreduce(k, C, n, dtype, op, inplace, with_status):
    assert torch.cuda.is_available()
    L = load_library()
    dist = {"fp32": "normal", "bf16": "normal", "fp16": "uniform", "int32": "int"}[dtype]
    kw = {"lo": -2 ** 20, "hi": 2 ** 20} if dtype == "int32" else {}
    xs = inputs.workload(91 + k * 7 + C, k, n, dtype, dist, **kw)
    sends = [to_dev(x) for x in xs]
    want = _reference(sends, k, C, dtype, op, inplace)

    status = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):       # two calls in a row share the scratch array
        srcs = [s.clone() for s in sends]
        outs = [srcs[r] if r in inplace else torch.full_like(s, 7) for r, s in enumerate(sends)]
        st = ctypes.c_void_p(status.data_ptr()) if with_status else None
        rc = L.vAllReduceNoAlloc(_ptrs(srcs), _ptrs(outs), n, DTYPE_CODES[dtype], OP_CODES[op],
                                 k, C, st, stream)
        assert RESULTS[rc] == "vSuccess"
        torch.cuda.synchronize()
        if with_status:
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
