"""LL128 line integrity under load.

The LL128 reader (Sec. III-C) polls only the flag word of a 128-byte line
(word 15, the upper 8 bytes of the line's last 16-byte piece) and then uses
the other seven 16-byte pieces it loaded in the same warp-wide load.  That is
correct only if the sender's one warp-wide 128-byte store of a line becomes
visible to the reader's one warp-wide 128-byte load as a whole: a line must
never be seen with its flag but with stale data in another piece.  The PTX
memory model does not state this; the protocol relies on the hardware
performing an aligned 128-byte warp access as one L2 transaction.

This test puts that assumption under stress: tiny FIFO slots (two or four
lines), so that every line is rewritten thousands of times per call; several
communicators on their own streams running at once; thousands of calls back
to back.  Every result is compared bit for bit with the oracle's.  A torn
line would show up as a wrong value (the flag of the new step beside data of
a step eight slots older).
"""
import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import Comm, inputs

from gpu_util import assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (vranks, channels, elements, dtype, algorithm, LL128 slot bytes)
COMMS = [(4, 3, 20_011, "fp32", "ring", 256),
         (5, 2, 17_333, "bf16", "ring", 512),
         (8, 2, 12_007, "fp32", "tree", 256),
         (3, 4, 9_001, "fp32", "ring", 256)]
CALLS = 1500      # per communicator
RING = 6          # output sets per communicator, checked every RING calls


def test_ll128_lines_stay_whole_under_load():
    setups = []
    for i, (k, C, n, dt, algo, slot) in enumerate(COMMS):
        sets = [inputs.workload(700 + 10 * i + j, k, n, dt, "normal") for j in range(2)]
        ch = chunk_for("ll128", dt, {"ll128": slot}, 1)
        want = [oracle.all_reduce(xs, dt, "sum", C, ch, algo) for xs in sets]
        c = Comm(k, C, slot_bytes={"ll128": slot}, timeout_sec=10.0)
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
                                   proto="ll128", stream=su["stream"])
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
        assert su["c"].last_plan()["proto"] == "ll128"
        su["c"].destroy()
    assert not bad
