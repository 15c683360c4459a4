"""ctypes binding of the C ABI in include/vcomm.h.

Argument marshalling only: every step of every collective runs in the CUDA
kernels of libvcomm.so.  Tensors are torch CUDA tensors; only their data
pointers and the stream handle cross the boundary.  There is no fallback: if
the library is missing, the first call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libvcomm.so")

RESULTS = {0: "vSuccess", 1: "vInvalidArgument", 2: "vUnsupported", 3: "vOutOfMemory",
           4: "vCudaError", 5: "vTimeout", 6: "vAborted", 7: "vInternalError"}
DTYPE_CODES = {"int32": 0, "fp32": 1, "fp16": 2, "bf16": 3, "int8": 4, "uint8": 5, "uint32": 6,
               "int64": 7, "uint64": 8, "fp64": 9}
OP_CODES = {"sum": 0, "max": 1, "prod": 2, "min": 3, "avg": 4}
ALGO_CODES = {"auto": 0, "ring": 1, "tree": 2}
PROTO_CODES = {"auto": 0, "simple": 1, "ll": 2, "ll128": 3, "cluster": 4, "direct": 5}
ALGO_NAMES = {v: k for k, v in ALGO_CODES.items()}
PROTO_NAMES = {v: k for k, v in PROTO_CODES.items()}

# the exported symbols of include/vcomm.h
EXPORTS = ("vcommInit", "vcommInitConfig", "vcommPrepare", "vcommDestroy", "vcommAbort",
           "vcommGetAsyncError", "vcommSetPlan", "vcommGetLastPlan", "vAllReduce",
           "vReduceScatter", "vAllGather", "vBroadcast", "vReduce", "vcommVersion",
           "vDebugEncode", "vDebugDecode", "vAllReduceNoAlloc", "vGroupStart", "vGroupEnd",
           "vcommGetGroupPlans", "vcommTune", "vcommGetTuneTable", "vcommDebugSetSkipRank",
           "vServeCreate", "vServeSubmit", "vServeQuery", "vServeRelease", "vServeGetStats",
           "vServeDestroy", "vSend", "vRecv", "vAllToAll", "vcommAbortPending", "vcommReset",
           "vDebugHopLatency", "vDebugTileGeometry")


class VcommError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        self.name = RESULTS.get(code, str(code))
        super().__init__(f"{what}: {self.name}")


class Config(ctypes.Structure):
    _fields_ = [("slotBytes", ctypes.c_size_t * 3), ("nsteps", ctypes.c_int),
                ("nthreads", ctypes.c_int), ("timeoutSec", ctypes.c_double),
                ("treeNodeSize", ctypes.c_int)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("maxRanks", ctypes.c_int), ("memBudget", ctypes.c_size_t),
                ("bigGangChannels", ctypes.c_int), ("smallGangs", ctypes.c_int),
                ("bigThreshold", ctypes.c_size_t), ("slotBytes", ctypes.c_size_t * 3),
                ("idleTimeoutSec", ctypes.c_double), ("threads", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("inflightBytes", ctypes.c_size_t), ("maxInflightBytes", ctypes.c_size_t)]


class Plan(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("proto", ctypes.c_int), ("nchannels", ctypes.c_int),
                ("chunkSteps", ctypes.c_int)]

    def as_dict(self):
        return {"algo": ALGO_NAMES[self.algo], "proto": PROTO_NAMES[self.proto],
                "nchannels": self.nchannels, "chunkSteps": self.chunkSteps}


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libvcomm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libvcomm.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(_LIB_PATH)
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.vcommInit.argtypes = [ctypes.POINTER(vp), i32, i32]
    L.vcommInitConfig.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(Config)]
    L.vcommPrepare.argtypes = [vp, ctypes.c_uint, ctypes.c_uint]
    L.vcommDestroy.argtypes = [vp]
    L.vcommAbort.argtypes = [vp]
    L.vcommGetAsyncError.argtypes = [vp, ctypes.POINTER(i32)]
    L.vcommSetPlan.argtypes = [vp, ctypes.POINTER(Plan)]
    L.vcommGetLastPlan.argtypes = [vp, ctypes.POINTER(Plan)]
    L.vAllReduce.argtypes = [pp, pp, sz, i32, i32, i32, i32, vp, vp]
    L.vReduceScatter.argtypes = [pp, pp, sz, i32, i32, i32, i32, vp, vp]
    L.vAllGather.argtypes = [pp, pp, sz, i32, i32, i32, vp, vp]
    L.vBroadcast.argtypes = [pp, pp, sz, i32, i32, i32, i32, vp, vp]
    L.vReduce.argtypes = [pp, pp, sz, i32, i32, i32, i32, i32, vp, vp]
    L.vcommVersion.argtypes = []
    L.vDebugEncode.argtypes = [i32, vp, sz, ctypes.c_uint64, vp, vp]
    L.vDebugDecode.argtypes = [i32, vp, sz, ctypes.c_uint64, vp, ctypes.c_double, vp]
    L.vAllReduceNoAlloc.argtypes = [pp, pp, sz, i32, i32, i32, i32, vp, vp]
    L.vcommDebugSetSkipRank.argtypes = [vp, i32]
    L.vDebugHopLatency.argtypes = [i32, ctypes.POINTER(i32), i32, i32, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
    L.vDebugTileGeometry.argtypes = [i32, i32, ctypes.c_uint64, i32, i32, ctypes.c_uint64, ctypes.c_uint64, i32,
                                     ctypes.POINTER(ctypes.c_uint64)]
    L.vServeCreate.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServeConfig)]
    L.vServeSubmit.argtypes = [vp, i32, pp, sz, i32, i32, i32, i32, i32, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_uint64)]
    L.vServeQuery.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(Plan), pp]
    L.vServeRelease.argtypes = [vp, ctypes.c_uint64]
    L.vServeGetStats.argtypes = [vp, ctypes.POINTER(ServeStats)]
    L.vServeDestroy.argtypes = [vp]
    L.vGroupStart.argtypes = []
    L.vGroupEnd.argtypes = []
    L.vcommGetGroupPlans.argtypes = [vp, ctypes.POINTER(Plan), i32, ctypes.POINTER(i32)]
    L.vcommTune.argtypes = [vp, ctypes.c_uint, sz, vp]
    L.vcommGetTuneTable.argtypes = [vp, i32, ctypes.POINTER(Plan), ctypes.POINTER(sz),
                                    ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(i32)]
    for name in EXPORTS:
        if name != "vcommVersion":
            getattr(L, name).restype = i32
    L.vcommVersion.restype = i32
    _lib = L
    return L


def version() -> int:
    return load_library().vcommVersion()


def _check(rc: int, what: str):
    if rc != 0:
        raise VcommError(rc, what)


def _dtype_name(t) -> str:
    import torch
    m = {torch.float32: "fp32", torch.float16: "fp16", torch.bfloat16: "bf16",
         torch.int32: "int32", torch.int8: "int8", torch.uint8: "uint8", torch.uint32: "uint32",
         torch.int64: "int64", torch.uint64: "uint64", torch.float64: "fp64"}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _ptr_array(ts):
    a = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        a[i] = None if t is None else (t if isinstance(t, int) else t.data_ptr())
    return a


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Comm:
    """A communicator of `nranks` virtual ranks on the current CUDA device."""

    def __init__(self, nranks: int, nchannels: int, slot_bytes=None, nsteps: int = 0,
                 nthreads: int = 0, timeout_sec: float = 0.0, tree_node: int = 0):
        L = load_library()
        self._h = ctypes.c_void_p()
        cfg = Config()
        if slot_bytes:
            for i, p in enumerate(("simple", "ll", "ll128")):
                cfg.slotBytes[i] = int(slot_bytes.get(p, 0))
        cfg.nsteps, cfg.nthreads, cfg.timeoutSec = nsteps, nthreads, timeout_sec
        cfg.treeNodeSize = tree_node
        _check(L.vcommInitConfig(ctypes.byref(self._h), nranks, nchannels, ctypes.byref(cfg)),
               "vcommInitConfig")
        self.nranks, self.nchannels = nranks, nchannels

    # -- lifetime
    def destroy(self):
        if self._h:
            _check(load_library().vcommDestroy(self._h), "vcommDestroy")
            self._h = ctypes.c_void_p()

    def abort_pending(self):
        """Raise the abort word; in-flight calls return early; the comm stays."""
        _check(load_library().vcommAbortPending(self._h), "vcommAbortPending")

    def reset(self):
        """Make a failed or aborted communicator usable again."""
        _check(load_library().vcommReset(self._h), "vcommReset")

    def abort(self):
        if self._h:
            _check(load_library().vcommAbort(self._h), "vcommAbort")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def prepare(self, algos=("ring",), protos=("simple",)):
        am = sum(1 << ALGO_CODES[a] for a in algos)
        pm = sum(1 << PROTO_CODES[p] for p in protos)
        _check(load_library().vcommPrepare(self._h, am, pm), "vcommPrepare")

    def async_error(self) -> str:
        e = ctypes.c_int()
        _check(load_library().vcommGetAsyncError(self._h, ctypes.byref(e)), "vcommGetAsyncError")
        return RESULTS[e.value]

    def set_plan(self, algo="auto", proto="auto", nchannels=0, chunk_steps=0):
        p = Plan(ALGO_CODES[algo], PROTO_CODES[proto], nchannels, chunk_steps)
        _check(load_library().vcommSetPlan(self._h, ctypes.byref(p)), "vcommSetPlan")

    def clear_plan(self):
        _check(load_library().vcommSetPlan(self._h, None), "vcommSetPlan")

    def last_plan(self) -> dict:
        p = Plan()
        _check(load_library().vcommGetLastPlan(self._h, ctypes.byref(p)), "vcommGetLastPlan")
        return p.as_dict()

    def debug_skip_rank(self, rank: int):
        _check(load_library().vcommDebugSetSkipRank(self._h, rank), "vcommDebugSetSkipRank")

    def group_plans(self) -> list:
        n = ctypes.c_int()
        arr = (Plan * 256)()
        _check(load_library().vcommGetGroupPlans(self._h, arr, 256, ctypes.byref(n)),
               "vcommGetGroupPlans")
        return [arr[i].as_dict() for i in range(min(n.value, 256))]

    def tune(self, colls=("allreduce",), max_bytes=64 << 20, stream=None):
        mask = sum(1 << COLL_BITS[c] for c in colls)
        _check(load_library().vcommTune(self._h, mask, max_bytes, _stream_handle(stream)),
               "vcommTune")

    def tune_table(self, coll="allreduce") -> list:
        n = ctypes.c_int()
        plans = (Plan * 32)()
        sizes = (ctypes.c_size_t * 32)()
        us = (ctypes.c_float * 32)()
        _check(load_library().vcommGetTuneTable(self._h, COLL_BITS[coll], plans, sizes, us, 32,
                                                ctypes.byref(n)), "vcommGetTuneTable")
        return [dict(plans[i].as_dict(), bytes=sizes[i], usec=us[i])
                for i in range(min(n.value, 32))]

    # -- collectives (lists of torch CUDA tensors, one per vrank)
    def all_reduce(self, sends, recvs, op="sum", algo="ring", proto="simple", stream=None,
                   count=None):
        dt = _dtype_name(sends[0])
        n = sends[0].numel() if count is None else count
        _check(load_library().vAllReduce(_ptr_array(sends), _ptr_array(recvs), n,
                                         DTYPE_CODES[dt], OP_CODES[op], ALGO_CODES[algo],
                                         PROTO_CODES[proto], _stream_handle(stream), self._h),
               "vAllReduce")

    def reduce_scatter(self, sends, recvs, op="sum", algo="ring", proto="simple", stream=None,
                       recvcount=None):
        dt = _dtype_name(sends[0])
        n = recvs[0].numel() if recvcount is None else recvcount
        _check(load_library().vReduceScatter(_ptr_array(sends), _ptr_array(recvs), n,
                                             DTYPE_CODES[dt], OP_CODES[op], ALGO_CODES[algo],
                                             PROTO_CODES[proto], _stream_handle(stream),
                                             self._h), "vReduceScatter")

    def all_gather(self, sends, recvs, algo="ring", proto="simple", stream=None,
                   sendcount=None):
        dt = _dtype_name(sends[0])
        n = sends[0].numel() if sendcount is None else sendcount
        _check(load_library().vAllGather(_ptr_array(sends), _ptr_array(recvs), n,
                                         DTYPE_CODES[dt], ALGO_CODES[algo], PROTO_CODES[proto],
                                         _stream_handle(stream), self._h), "vAllGather")

    def broadcast(self, sends, recvs, root=0, algo="ring", proto="simple", stream=None,
                  count=None):
        ref = sends[root] if 0 <= root < len(sends) and sends[root] is not None else recvs[0]
        dt = _dtype_name(ref)
        n = recvs[0].numel() if count is None else count
        _check(load_library().vBroadcast(_ptr_array(sends), _ptr_array(recvs), n,
                                         DTYPE_CODES[dt], root, ALGO_CODES[algo],
                                         PROTO_CODES[proto], _stream_handle(stream), self._h),
               "vBroadcast")

    def send(self, rank, peer, tensor, count=None, stream=None):
        """vrank `rank` sends `tensor` to vrank `peer` (inside a group)."""
        n = tensor.numel() if count is None else count
        _check(load_library().vSend(ctypes.c_void_p(tensor.data_ptr()), n,
                                    DTYPE_CODES[_dtype_name(tensor)], rank, peer, self._h,
                                    _stream_handle(stream)), "vSend")

    def recv(self, rank, peer, tensor, count=None, stream=None):
        """vrank `rank` receives into `tensor` from vrank `peer` (inside a group)."""
        n = tensor.numel() if count is None else count
        _check(load_library().vRecv(ctypes.c_void_p(tensor.data_ptr()), n,
                                    DTYPE_CODES[_dtype_name(tensor)], rank, peer, self._h,
                                    _stream_handle(stream)), "vRecv")

    def all_to_all(self, sends, recvs, count=None, stream=None):
        """Block j of sends[r] lands in block r of recvs[j]."""
        k = len(sends)
        n = sends[0].numel() // k if count is None else count
        _check(load_library().vAllToAll(_ptr_array(sends), _ptr_array(recvs), n,
                                        DTYPE_CODES[_dtype_name(sends[0])], self._h,
                                        _stream_handle(stream)), "vAllToAll")

    def reduce(self, sends, recvs, op="sum", root=0, algo="ring", proto="simple", stream=None,
               count=None):
        dt = _dtype_name(sends[0])
        n = sends[0].numel() if count is None else count
        _check(load_library().vReduce(_ptr_array(sends), _ptr_array(recvs), n, DTYPE_CODES[dt],
                                      OP_CODES[op], root, ALGO_CODES[algo], PROTO_CODES[proto],
                                      _stream_handle(stream), self._h), "vReduce")


COLL_BITS = {"allreduce": 0, "reducescatter": 1, "allgather": 2, "broadcast": 3, "reduce": 4}


def group_start():
    _check(load_library().vGroupStart(), "vGroupStart")


def group_end():
    _check(load_library().vGroupEnd(), "vGroupEnd")


class group:
    """Context manager: collectives issued inside run as one batched launch
    per communicator at exit (vGroupStart / vGroupEnd)."""

    def __enter__(self):
        group_start()
        return self

    def __exit__(self, exc_type, *a):
        if exc_type is None:
            group_end()
        else:
            try:
                group_end()
            except VcommError:
                pass
        return False


SERVE_COLLS = {"allreduce": 0, "reducescatter": 1, "allgather": 2}
SERVE_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class Server:
    """Continuous-batching server of collective requests (vServe* in vcomm.h).
    mode: "streams" (concurrent launches on lanes of streams), "batch" (a
    resident gang kernel fed through mailboxes), "tiles" (a resident kernel
    whose CTAs take tiles of direct-protocol requests, small ones first) or
    "plain" (one launch per request on one stream, for comparison)."""

    def __init__(self, mode="batch", max_ranks=16, mem_budget=40 << 30, big_gang_channels=0,
                 small_gangs=1, big_threshold=4 << 20, slot_bytes=None, idle_timeout_sec=30.0,
                 threads=512):
        L = load_library()
        cfg = ServeConfig()
        cfg.mode = {"batch": 0, "plain": 1, "streams": 2, "tiles": 3}[mode]
        cfg.maxRanks = max_ranks
        cfg.memBudget = mem_budget
        cfg.bigGangChannels = big_gang_channels
        cfg.smallGangs = small_gangs
        cfg.bigThreshold = big_threshold
        if slot_bytes:
            for i, p in enumerate(("simple", "ll", "ll128")):
                cfg.slotBytes[i] = int(slot_bytes.get(p, 0))
        cfg.idleTimeoutSec = idle_timeout_sec
        cfg.threads = threads
        self._h = ctypes.c_void_p()
        _check(L.vServeCreate(ctypes.byref(self._h), ctypes.byref(cfg)), "vServeCreate")

    def submit(self, coll, sends, count, dtype, op="sum", proto="auto", release=False,
               arrival_ns=0) -> int:
        t = ctypes.c_uint64()
        _check(load_library().vServeSubmit(self._h, SERVE_COLLS[coll], _ptr_array(sends), count,
                                           DTYPE_CODES[dtype], OP_CODES[op], len(sends),
                                           PROTO_CODES[proto], 1 if release else 0, arrival_ns,
                                           ctypes.byref(t)), "vServeSubmit")
        return t.value

    def query(self, ticket, nranks=16):
        """(state, latency ns, plan, receive buffers)"""
        st, lat, svc, plan = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64(), Plan()
        bufs = (ctypes.c_void_p * nranks)()
        _check(load_library().vServeQuery(self._h, ticket, ctypes.byref(st), ctypes.byref(lat),
                                          ctypes.byref(svc), ctypes.byref(plan), bufs),
               "vServeQuery")
        self.last_service_ns = svc.value
        return (SERVE_STATES[st.value], lat.value, plan.as_dict(),
                [bufs[i] for i in range(nranks)])

    def release(self, ticket):
        _check(load_library().vServeRelease(self._h, ticket), "vServeRelease")

    def stats(self) -> dict:
        st = ServeStats()
        _check(load_library().vServeGetStats(self._h, ctypes.byref(st)), "vServeGetStats")
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}

    def destroy(self):
        if self._h:
            _check(load_library().vServeDestroy(self._h), "vServeDestroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def debug_hop_latency(proto: str, sms=None, n: int = 0, laps: int = 1000, timeout_sec: float = 2.0):
    """(ns per hop, SM id of each ring position) of a ring of CTAs passing one
    FIFO line (vDebugHopLatency): `sms` lists the ring's SM ids, or None for
    one cluster of n CTAs."""
    if sms is not None:
        n = len(sms)
        arr = (ctypes.c_int * n)(*sms)
    else:
        arr = None
    ns = ctypes.c_double()
    out = (ctypes.c_int * n)()
    _check(load_library().vDebugHopLatency(PROTO_CODES[proto], arr, n, laps, ctypes.c_double(timeout_sec),
                                           ctypes.byref(ns), out), "vDebugHopLatency")
    return ns.value, list(out)


TILE_COLLS = {"allreduce": 0, "reducescatter": 1, "allgather": 2, "broadcast": 3, "reduce": 4}


def debug_tile_geometry(coll: str, nranks: int, count: int, dtype_size: int, vec: int,
                        workers: int = 147, iter_units: int = 256, shared: bool = False) -> dict:
    """The tiles the tile engine cuts a direct-protocol op into
    (vDebugTileGeometry; host arithmetic, no device); shared: for a group
    launch (tiles shared out statically) rather than serving."""
    out = (ctypes.c_uint64 * 8)()
    _check(load_library().vDebugTileGeometry(TILE_COLLS[coll], nranks, count, dtype_size, vec, workers,
                                             iter_units, int(shared), out), "vDebugTileGeometry")
    keys = ("staged", "units", "tileUnits", "blockBytes", "tileBytes", "perBlock", "ntiles", "vec")
    return dict(zip(keys, [int(v) for v in out]))


def debug_encode(proto: str, src, nbytes: int, flag: int, lines, stream=None):
    _check(load_library().vDebugEncode(PROTO_CODES[proto], src.data_ptr(), nbytes, flag,
                                       lines.data_ptr(), _stream_handle(stream)), "vDebugEncode")


def debug_decode(proto: str, lines, nbytes: int, flag: int, dst, timeout_sec: float = 1.0,
                 stream=None) -> str:
    rc = load_library().vDebugDecode(PROTO_CODES[proto], lines.data_ptr(), nbytes, flag,
                                     dst.data_ptr(), timeout_sec, _stream_handle(stream))
    return RESULTS[rc]
