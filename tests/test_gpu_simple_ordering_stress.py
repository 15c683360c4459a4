"""Simple and LL FIFO publication order under load.

A Simple step (Sec. III-A) publishes its slot without a fence in every
thread: the step's threads write the slot, meet at the block barrier, and
thread 0 alone issues one release fence and then advances the connection
counters with relaxed stores (the send's tail, the receive's head).  The
receiver's thread 0 acquires the tail and its block barrier comes before any
thread reads the slot.  The barrier orders every thread's slot writes before
thread 0's fence, and the fence's cumulativity carries them to device scope;
a mistake in that chain would let a receiver read a slot before all of its
bytes had landed, or let a sender overwrite a slot still being read.

LL (Sec. III-B) returns its slots the same way but without the fence: its
data is published by the lines' flags, and the receiver's head is a relaxed
store after the barrier that follows the step's reads.  Both protocols run
here.

This test puts the chain under stress: the smallest slots the library takes
(256 and 512 bytes, so a call takes hundreds of steps), FIFOs of 2, 3 and 8
slots (the credit counters gate almost every step), ring and tree workers,
several communicators on their own streams at once, and hundreds of calls
back to back.  Every output is compared bit for bit with the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (vranks, channels, elements, dtype, algorithm, Simple slot bytes, slots per FIFO)
COMMS = [(4, 3, 20_011, "fp32", "ring", 256, 8),
         (5, 2, 17_333, "bf16", "ring", 512, 2),
         (8, 2, 12_007, "fp32", "tree", 256, 3),
         (16, 1, 5_003, "fp32", "ring", 256, 8)]
CALLS = 400       # per communicator
RING = 4          # output sets per communicator, checked every RING calls


@pytest.mark.parametrize("proto", ["simple", "ll"])
def test_slots_publish_in_order_under_load(proto):
    setups = []
    for i, (k, C, n, dt, algo, slot, ns) in enumerate(COMMS):
        sets = [inputs.workload(900 + 10 * i + j, k, n, dt, "normal") for j in range(2)]
        ch = chunk_for(proto, dt, {proto: slot}, 1)
        want = [oracle.all_reduce(xs, dt, "sum", C, ch, algo) for xs in sets]
        c = Comm(k, C, slot_bytes={proto: slot}, nsteps=ns, timeout_sec=10.0)
        c.set_plan(nchannels=C, chunk_steps=1)
        dev_in = [[to_dev(x) for x in xs] for xs in sets]
        dev_want = [[to_dev(w) for w in ws] for ws in want]
        outs = [[torch.empty_like(dev_in[0][0]) for _ in range(k)] for _ in range(RING)]
        setups.append(dict(c=c, algo=algo, dt=dt, k=k, ins=dev_in, want=dev_want, host_want=want,
                           outs=outs, stream=torch.cuda.Stream()))
    torch.cuda.synchronize()
    bad = []
    for it in range(CALLS):
        for su in setups:
            with torch.cuda.stream(su["stream"]):
                su["c"].all_reduce(su["ins"][it % 2], su["outs"][it % RING], op="sum", algo=su["algo"],
                                   proto=proto, stream=su["stream"])
        if it % RING == RING - 1:
            torch.cuda.synchronize()
            for ci, su in enumerate(setups):
                assert su["c"].async_error() == "vSuccess"
                for j in range(RING):
                    call = it - (RING - 1) + j
                    for r in range(su["k"]):
                        got, want = su["outs"][j][r], su["want"][call % 2][r]
                        if not torch.equal(got.view(torch.int16), want.view(torch.int16)):
                            bad.append((ci, call, r))
            if bad:
                break
            for su in setups:
                with torch.cuda.stream(su["stream"]):
                    for o in su["outs"]:
                        for t in o:
                            t.fill_(0)
    torch.cuda.synchronize()
    if bad:
        ci, call, r = bad[0]
        su = setups[ci]
        assert_same(to_np(su["outs"][call % RING][r], su["dt"]), su["host_want"][call % 2][r],
                    f"communicator {ci} call {call} rank {r} ({len(bad)} bad outputs)")
    for su in setups:
        assert su["c"].last_plan()["proto"] == proto
        su["c"].destroy()
    assert not bad
