"""CPU oracle for the virtual-rank collectives (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The arithmetic lives in ``vcomm_oracle.c`` (plain C loops, compiled with gcc,
no fast-math, no FP contraction).  This module only marshals numpy arrays.
Each function cites the passage of "Demystifying NCCL" (arXiv 2507.04786) it
models; the readings taken where the paper is silent are listed at the top of
the C file.

Dtypes are named 'int8', 'uint8', 'int32', 'uint32', 'int64', 'uint64', 'fp16',
'bf16', 'fp32', 'fp64'; ops 'sum', 'prod', 'max', 'min', 'avg'.  bf16 arrays
are carried as numpy uint16 bit patterns; fp16 arrays may be numpy float16 or
uint16 bits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vcomm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPES = {"int32": 0, "fp32": 1, "fp16": 2, "bf16": 3, "int8": 5, "uint8": 6, "uint32": 7,
          "int64": 8, "uint64": 9, "fp64": 10}
ESIZE = {"int32": 4, "fp32": 4, "fp16": 2, "bf16": 2, "int8": 1, "uint8": 1, "uint32": 4,
         "int64": 8, "uint64": 8, "fp64": 8}
OPS = {"sum": 0, "max": 1, "prod": 2, "min": 3, "avg": 4}
PROTOS = {"simple": 0, "ll": 1, "ll128": 2}
PRIMS = {0: None, 1: "send", 2: "recv", 3: "recvReduceSend", 4: "recvCopySend",
         5: "recvReduceCopySend", 6: "copySend", 7: "recvReduceCopy"}

# Table "buffer sizes" (Sec. V-C): default per-slot buffer bytes, 8 slots per channel
DEFAULT_SLOT_BYTES = {"simple": 512 * 1024, "ll": 32 * 1024, "ll128": 600 * 1024}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        sz, i32, vp = ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.o_chunk_units.restype = sz
        L.o_chunk_units.argtypes = [i32, sz, i32, i32]
        L.o_slot_data_bytes.restype = sz
        L.o_slot_data_bytes.argtypes = [i32, sz]
        L.o_channel_range.argtypes = [sz, i32, i32, i32, ctypes.POINTER(sz), ctypes.POINTER(sz)]
        L.o_ring_loop_chunk.restype = sz
        L.o_ring_loop_chunk.argtypes = [sz, sz, i32, sz, i32]
        for f in ("o_ring_allreduce_prim", "o_ring_reducescatter_prim"):
            getattr(L, f).argtypes = [i32, i32]
        L.o_ring_allgather_prim.argtypes = [i32, i32, i32]
        L.o_bcast_prim.argtypes = [i32, i32, i32, i32]
        L.o_reduce_prim.argtypes = [i32, i32, i32]
        L.o_tree_links.argtypes = [i32, i32, i32] + [ctypes.POINTER(i32)] * 3
        L.o_tree_root.argtypes = [i32, i32]
        L.o_htree_links.argtypes = [i32, i32, i32, i32] + [ctypes.POINTER(i32)] * 3
        L.o_htree_root.argtypes = [i32, i32, i32]
        L.o_tree_prims.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.o_ring_allreduce.argtypes = [i32, i32, sz, i32, i32, sz, pp, pp]
        L.o_ring_reducescatter.argtypes = [i32, i32, sz, i32, i32, sz, pp, pp]
        L.o_ring_allgather.argtypes = [i32, i32, sz, sz, pp, pp]
        L.o_ring_broadcast.argtypes = [i32, i32, sz, sz, i32, pp, pp]
        L.o_alltoall.argtypes = [i32, sz, pp, pp]
        L.o_ring_reduce.argtypes = [i32, i32, sz, i32, i32, sz, i32, pp, pp]
        L.o_tree_allreduce.argtypes = [i32, i32, sz, i32, i32, sz, pp, pp]
        L.o_tree_allreduce_m.argtypes = [i32, i32, i32, sz, i32, i32, sz, pp, pp]
        L.o_tree_allreduce_point_m.argtypes = [i32, i32, i32, sz, i32, i32, sz, sz, vp, vp]
        L.o_encode_array.argtypes = [i32, vp, sz, vp]
        L.o_decode_array.argtypes = [i32, vp, sz, vp]
        L.o_ll_lines.restype = sz
        L.o_ll_lines.argtypes = [sz]
        L.o_ll128_lines.restype = sz
        L.o_ll128_lines.argtypes = [sz]
        L.o_ll_encode.argtypes = [vp, sz, ctypes.c_uint32, vp]
        L.o_ll_decode.restype = ctypes.c_long
        L.o_ll_decode.argtypes = [vp, sz, ctypes.c_uint32, vp]
        L.o_ll128_encode.argtypes = [vp, sz, ctypes.c_uint64, vp]
        L.o_ll128_decode.restype = ctypes.c_long
        L.o_ll128_decode.argtypes = [vp, sz, ctypes.c_uint64, vp]
        for f in ("o_ring_allreduce_point", "o_tree_allreduce_point"):
            getattr(L, f).argtypes = [i32, i32, sz, i32, i32, sz, sz, vp, vp]
        L.o_ring_reducescatter_point.argtypes = [i32, i32, i32, i32, vp, vp]
        L.o_ring_reduce_point.argtypes = [i32, i32, i32, i32, vp, vp]
        L.o_f64_to_f16.restype = ctypes.c_uint16
        L.o_f64_to_f16.argtypes = [ctypes.c_double]
        L.o_f64_to_bf16.restype = ctypes.c_uint16
        L.o_f64_to_bf16.argtypes = [ctypes.c_double]
        L.o_f64_to_f32bits.restype = ctypes.c_uint32
        L.o_f64_to_f32bits.argtypes = [ctypes.c_double]
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers

def _ptrs(arrs):
    a = (ctypes.c_void_p * len(arrs))()
    for i, x in enumerate(arrs):
        a[i] = None if x is None else x.ctypes.data
    return a


def _raw(x: np.ndarray) -> np.ndarray:
    """contiguous view as raw bytes-compatible array (keeps itemsize)"""
    return np.ascontiguousarray(x)


def _unit_bytes(dtype: str) -> int:
    return ESIZE[dtype]


# ---------------------------------------------------------------- partition

def slot_data_bytes(proto: str, slot_bytes: int | None = None) -> int:
    """Effective data per slot (Table "buffer sizes")."""
    sb = DEFAULT_SLOT_BYTES[proto] if slot_bytes is None else slot_bytes
    return int(lib().o_slot_data_bytes(PROTOS[proto], sb))


def chunk_units(proto: str, unit_bytes: int, chunk_steps: int = 1,
                slot_bytes: int | None = None) -> int:
    """chunkCount (Sec. V-C) in units of `unit_bytes` for one elementary step."""
    sb = DEFAULT_SLOT_BYTES[proto] if slot_bytes is None else slot_bytes
    return int(lib().o_chunk_units(PROTOS[proto], sb, chunk_steps, unit_bytes))


def channel_range(n: int, unit_bytes: int, nch: int, ch: int):
    """(workOffset, channelCount) of channel `ch` (Sec. V-C, reading R1)."""
    s, l = ctypes.c_size_t(), ctypes.c_size_t()
    lib().o_channel_range(n, unit_bytes, nch, ch, ctypes.byref(s), ctypes.byref(l))
    return s.value, l.value


def ring_loop_chunk(off: int, end: int, k: int, chunk: int, unit_bytes: int) -> int:
    return int(lib().o_ring_loop_chunk(off, end, k, chunk, unit_bytes))


# ---------------------------------------------------------------- step tables

def ring_prim(coll: str, k: int, t: int, inplace: bool = False):
    L = lib()
    if coll == "allreduce":
        return PRIMS[L.o_ring_allreduce_prim(k, t)]
    if coll == "reducescatter":
        return PRIMS[L.o_ring_reducescatter_prim(k, t)]
    if coll == "allgather":
        return PRIMS[L.o_ring_allgather_prim(k, t, int(inplace))]
    raise ValueError(coll)


def chain_prim(coll: str, k: int, root: int, r: int, inplace: bool = False):
    L = lib()
    if coll == "broadcast":
        return PRIMS[L.o_bcast_prim(k, root, r, int(inplace))]
    if coll == "reduce":
        return PRIMS[L.o_reduce_prim(k, root, r)]
    raise ValueError(coll)


def tree_links(k: int, t: int, r: int):
    p, c0, c1 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().o_tree_links(k, t, r, ctypes.byref(p), ctypes.byref(c0), ctypes.byref(c1))
    return p.value, c0.value, c1.value


def tree_root(k: int, t: int) -> int:
    return int(lib().o_tree_root(k, t))


def htree_links(k: int, m: int, t: int, r: int):
    """(parent, child0, child1) of rank r in tree t of the hierarchical tree
    with nodes of m ranks (Sec. V-E, reading R19); -1 for none."""
    p, c0, c1 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().o_htree_links(k, m, t, r, ctypes.byref(p), ctypes.byref(c0), ctypes.byref(c1))
    return p.value, c0.value, c1.value


def htree_root(k: int, m: int, t: int) -> int:
    return int(lib().o_htree_root(k, m, t))


def tree_prims(k: int, t: int, r: int):
    u, d = ctypes.c_int(), ctypes.c_int()
    lib().o_tree_prims(k, t, r, ctypes.byref(u), ctypes.byref(d))
    return PRIMS[u.value], PRIMS[d.value]


# ---------------------------------------------------------------- dtype codecs

def encode(dtype: str, x) -> np.ndarray:
    """Round fp64 values to `dtype` (own IEEE round-to-nearest-even).
    Returns float32 / float16 arrays, or uint16 bit patterns for bf16."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if dtype == "fp32":
        out = np.empty(x.shape, np.float32)
    elif dtype == "fp16":
        out = np.empty(x.shape, np.float16)
    elif dtype == "bf16":
        out = np.empty(x.shape, np.uint16)
    else:
        raise ValueError(dtype)
    lib().o_encode_array(DTYPES[dtype], x.ctypes.data, x.size, out.ctypes.data)
    return out


def decode(dtype: str, x: np.ndarray) -> np.ndarray:
    """Exact widening of `dtype` values to fp64."""
    x = np.ascontiguousarray(x)
    out = np.empty(x.shape, np.float64)
    lib().o_decode_array(DTYPES[dtype], x.ctypes.data, x.size, out.ctypes.data)
    return out


# ---------------------------------------------------------------- collectives

def _check(xs, n, dtype):
    es = ESIZE[dtype]
    for x in xs:
        assert x.flags.c_contiguous and x.nbytes == n * es, (x.nbytes, n, es)


def _np_dtype(dtype):
    return {"int32": np.int32, "fp32": np.float32, "fp16": np.float16, "bf16": np.uint16,
            "int8": np.int8, "uint8": np.uint8, "uint32": np.uint32, "int64": np.int64,
            "uint64": np.uint64, "fp64": np.float64}[dtype]


def all_reduce(xs, dtype: str, op: str, nch: int, chunk: int, algo: str = "ring", node: int = 1):
    """Ring AllReduce (Table "Ring AllReduce") or double-binary-tree AllReduce
    (Table "Tree AllReduce"); `node` > 1: the hierarchical tree with chains of
    `node` ranks inside each node (Sec. V-E).  `chunk` is chunkCount in
    elements."""
    xs = [_raw(x) for x in xs]
    k, n = len(xs), xs[0].size
    _check(xs, n, dtype)
    outs = [np.empty_like(xs[0]) for _ in range(k)]
    if algo == "ring":
        rc = lib().o_ring_allreduce(k, nch, chunk, DTYPES[dtype], OPS[op], n, _ptrs(xs), _ptrs(outs))
    else:
        rc = lib().o_tree_allreduce_m(k, node, nch, chunk, DTYPES[dtype], OPS[op], n, _ptrs(xs),
                                      _ptrs(outs))
    assert rc == 0
    return outs


def reduce_scatter(xs, dtype: str, op: str, nch: int, chunk: int):
    """Ring ReduceScatter (Table "Ring ReduceScatter"): xs[r] holds k blocks."""
    xs = [_raw(x) for x in xs]
    k = len(xs)
    assert xs[0].size % k == 0
    rc_ = xs[0].size // k
    outs = [np.empty(rc_, dtype=xs[0].dtype) for _ in range(k)]
    rc = lib().o_ring_reducescatter(k, nch, chunk, DTYPES[dtype], OPS[op], rc_, _ptrs(xs),
                                    _ptrs(outs))
    assert rc == 0
    return outs


def all_gather(xs, nch: int, chunk_bytes: int):
    """Ring AllGather (Table "Ring AllGather"), byte units (Sec. V-C)."""
    xs = [_raw(x) for x in xs]
    k = len(xs)
    nb = xs[0].nbytes
    outs = [np.empty(k * xs[0].size, dtype=xs[0].dtype) for _ in range(k)]
    rc = lib().o_ring_allgather(k, nch, chunk_bytes, nb, _ptrs(xs), _ptrs(outs))
    assert rc == 0
    return outs


def broadcast(xs, root: int, nch: int, chunk_bytes: int):
    """Ring Broadcast chain (Table "Ring Broadcast"), byte units."""
    xs = [_raw(x) for x in xs]
    k = len(xs)
    outs = [np.empty_like(xs[0]) for _ in range(k)]
    rc = lib().o_ring_broadcast(k, nch, chunk_bytes, xs[0].nbytes, root, _ptrs(xs), _ptrs(outs))
    assert rc == 0
    return outs


def all_to_all(xs):
    """All-to-all (Sec. II-A-4, the grouped Send/Recv pattern): block j of
    rank r's input (len / k elements) becomes block r of rank j's output."""
    xs = [np.ascontiguousarray(x) for x in xs]
    k = len(xs)
    assert xs[0].size % k == 0
    outs = [np.empty_like(xs[0]) for _ in range(k)]
    rc = lib().o_alltoall(k, xs[0].nbytes // k, _ptrs(xs), _ptrs(outs))
    assert rc == 0
    return outs


def p2p_match(sends, recvs):
    """Point-to-point transfers of one group (Sec. II-A-3): sends is a list of
    (rank, peer, array) in issue order, recvs a list of (rank, peer, count);
    the i-th send from a to b meets the i-th receive at b from a.  Returns the
    array each receive gets, in recvs order; raises ValueError on an
    unmatched or mismatched transfer."""
    from collections import defaultdict, deque
    q = defaultdict(deque)
    for a, b, x in sends:
        q[(a, b)].append(np.ascontiguousarray(x))
    out = []
    for b, a, n in recvs:
        if not q[(a, b)]:
            raise ValueError(f"receive at {b} from {a} has no send")
        x = q[(a, b)].popleft()
        if x.size != n:
            raise ValueError(f"send {a}->{b} of {x.size} elements meets a receive of {n}")
        out.append(x.copy())
    if any(q[key] for key in q):
        raise ValueError("a send has no receive")
    return out


def reduce(xs, dtype: str, op: str, root: int, nch: int, chunk: int):
    """Ring Reduce chain (Table "Ring Reduce"); returns the root's output."""
    xs = [_raw(x) for x in xs]
    k, n = len(xs), xs[0].size
    outs = [None] * k
    outs[root] = np.empty_like(xs[0])
    rc = lib().o_ring_reduce(k, nch, chunk, DTYPES[dtype], OPS[op], n, root, _ptrs(xs),
                             _ptrs(outs))
    assert rc == 0
    return outs[root]


# ---------------------------------------------------------------- encodings

def ll_encode(data: bytes | np.ndarray, flag: int) -> np.ndarray:
    """LL lines (Sec. III-B): (flag << 32) | 4 data bytes."""
    d = np.frombuffer(bytes(data), np.uint8) if not isinstance(data, np.ndarray) else \
        np.ascontiguousarray(data).view(np.uint8).ravel()
    nl = int(lib().o_ll_lines(d.size))
    out = np.zeros(nl, np.uint64)
    lib().o_ll_encode(d.ctypes.data, d.size, flag, out.ctypes.data)
    return out


def ll_decode(lines: np.ndarray, nbytes: int, flag: int):
    """Returns (status, bytes): status 0 or 1 + first line with a stale flag."""
    lines = np.ascontiguousarray(lines, dtype=np.uint64)
    out = np.zeros(nbytes, np.uint8)
    st = lib().o_ll_decode(lines.ctypes.data, nbytes, flag, out.ctypes.data)
    return int(st), out


def ll128_encode(data, flag: int) -> np.ndarray:
    """LL128 lines (Sec. III-C): 120 data bytes + 8-byte flag per 128 bytes."""
    d = np.frombuffer(bytes(data), np.uint8) if not isinstance(data, np.ndarray) else \
        np.ascontiguousarray(data).view(np.uint8).ravel()
    nl = int(lib().o_ll128_lines(d.size))
    out = np.zeros(16 * nl, np.uint64)
    lib().o_ll128_encode(d.ctypes.data, d.size, flag, out.ctypes.data)
    return out


def ll128_decode(lines: np.ndarray, nbytes: int, flag: int):
    lines = np.ascontiguousarray(lines, dtype=np.uint64)
    out = np.zeros(nbytes, np.uint8)
    st = lib().o_ll128_decode(lines.ctypes.data, nbytes, flag, out.ctypes.data)
    return int(st), out


def all_reduce_points(xs, idx, dtype: str, op: str, nch: int, chunk: int, algo: str = "ring",
                      node: int = 1):
    """Elements `idx` of the AllReduce result, computed one at a time (for
    outputs too large to replay whole).  xs: per-rank inputs (numpy arrays of
    the full length, or equivalently any arrays whose [idx] are the values)."""
    L = lib()
    k = len(xs)
    if algo == "ring":
        f = L.o_ring_allreduce_point
    else:
        def f(k_, nch_, chunk_, dt_, op_, n_, i_, v_, o_):
            return L.o_tree_allreduce_point_m(k_, node, nch_, chunk_, dt_, op_, n_, i_, v_, o_)
    n = xs[0].size
    out = np.empty(len(idx), dtype=xs[0].dtype)
    vals = np.empty(k, dtype=xs[0].dtype)
    one = np.empty(1, dtype=xs[0].dtype)
    for m, i in enumerate(idx):
        for r in range(k):
            vals[r] = xs[r][i]
        rc = f(k, nch, chunk, DTYPES[dtype], OPS[op], n, int(i), vals.ctypes.data, one.ctypes.data)
        assert rc == 0
        out[m] = one[0]
    return out


def _fold_points(f, xs, idx, dtype, op, extra, offset=0):
    k = len(xs)
    out = np.empty(len(idx), dtype=xs[0].dtype)
    vals = np.empty(k, dtype=xs[0].dtype)
    one = np.empty(1, dtype=xs[0].dtype)
    for m, i in enumerate(idx):
        for r in range(k):
            vals[r] = xs[r][offset + i]
        assert f(k, DTYPES[dtype], OPS[op], extra, vals.ctypes.data, one.ctypes.data) == 0
        out[m] = one[0]
    return out


def reduce_scatter_points(xs, b, idx, dtype: str, op: str):
    """Elements `idx` of rank b's ReduceScatter output (block b), one at a time."""
    n = xs[0].size // len(xs)
    return _fold_points(lib().o_ring_reducescatter_point, xs, idx, dtype, op, b, offset=b * n)


def reduce_points(xs, root: int, idx, dtype: str, op: str):
    """Elements `idx` of the Reduce result at `root`, one at a time."""
    return _fold_points(lib().o_ring_reduce_point, xs, idx, dtype, op, root)
