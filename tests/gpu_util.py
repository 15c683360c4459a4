"""Helpers shared by the GPU tests: numpy <-> torch transfers and oracle plans."""
import numpy as np

import oracle

ESZ = {"int32": 4, "fp32": 4, "fp16": 2, "bf16": 2, "int8": 1, "uint8": 1, "uint32": 4, "int64": 8,
       "uint64": 8, "fp64": 8}

# small FIFO slots so that modest sizes span many loops, chunks and FIFO steps
SMALL_SLOTS = {"simple": 8192, "ll": 2048, "ll128": 2560}


def to_dev(x, dev="cuda"):
    import torch
    if x.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int16)).to(dev).view(torch.bfloat16)
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def to_np(t, dtype):
    import torch
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    out = t.cpu().numpy()
    want = {"int32": np.int32, "fp32": np.float32, "fp16": np.float16, "int8": np.int8,
            "uint8": np.uint8, "uint32": np.uint32, "int64": np.int64, "uint64": np.uint64,
            "fp64": np.float64}[dtype]
    return out.astype(want, copy=False)


def bits(a):
    return np.ascontiguousarray(a).view(np.uint8)


# The cluster protocol moves LL lines through FIFOs of fixed 8 KiB slots: to
# the oracle it is LL with that slot size.  The direct protocol takes its
# segments from the Simple protocol's chunk.
CLUSTER_SLOT_BYTES = 8192


def chunk_for(proto, dtype, slots=None, chunk_steps=1, byte_units=False):
    ub = 1 if byte_units else ESZ[dtype]
    if proto == "cluster":
        return oracle.chunk_units("ll", ub, chunk_steps, CLUSTER_SLOT_BYTES)
    if proto == "direct":
        proto = "simple"
    sb = None if slots is None else slots[proto]
    return oracle.chunk_units(proto, ub, chunk_steps, sb)


def assert_same(got, want, what=""):
    g, w = bits(got), bits(want)
    if not np.array_equal(g, w):
        gi = np.ascontiguousarray(got).ravel()
        wi = np.ascontiguousarray(want).ravel()
        diff = np.nonzero((bits(gi).reshape(gi.size, -1) != bits(wi).reshape(wi.size, -1)).any(axis=1))[0]
        raise AssertionError(f"{what}: {diff.size} of {gi.size} elements differ, first at "
                             f"{diff[:8].tolist()}: got {gi[diff[:4]]} want {wi[diff[:4]]}")
