"""Benchmark: 8-vrank ring AllReduce, 256 MiB per vrank, fp32 sum, on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--proto simple|ll128|ll] [--sweep out.jsonl]

One step = one AllReduce over the 8 virtual ranks (one kernel launch).  Prints
ONE JSON line: bus bandwidth (nccl-tests convention: algbw * 2(k-1)/k) of the
whole job, the HBM roofline of the kernel (algorithmic bytes 2kS + 4(k-1)S f,
f = 1 Simple, 2 LL, 128/120 LL128, over the measured HBM copy bandwidth), the
end-to-end figure through the C ABI with host buffers, the CPU oracle on a
bounded sample, and the SM clocks sampled during the timed region.

Under torchrun (--gpus N > 1) every rank runs its own replica on its own GPU
(the collectives never leave one GPU); the value is the total over ranks
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_04786_b300 import inputs, workloads  # noqa: E402

# FIFO bytes in HBM per data byte; the cluster protocol's FIFOs are in shared
# memory and the direct protocol has none
FIFO_FACTOR = {"simple": 1.0, "ll": 2.0, "ll128": 128.0 / 120.0, "cluster": 0.0, "direct": 0.0}


def algorithmic_bytes(k, S, proto):
    """System-wide bytes of a k-vrank ring AllReduce of S bytes per vrank:
    user 2kS (read inputs, write outputs) + FIFO 2 * 2(k-1)S * f."""
    return 2 * k * S + 4 * (k - 1) * S * FIFO_FACTOR[proto]


def busbw(S, k, seconds):
    return S / seconds * 2 * (k - 1) / k / 1e9


# B300 nominal HBM3e bandwidth (GB/s): the ~8 TB/s the part is quoted at,
# reported beside the measured copy bandwidth as a second denominator
NOMINAL_HBM_GBS = 8000.0


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# the sources the reducing collective kernel (kReduceColl) is compiled from
KERNEL_SOURCES = ("include/vcomm.h", "paper_2507_04786_b300/csrc/vcomm_device.cuh",
                  "paper_2507_04786_b300/csrc/vcomm_internal.h",
                  "paper_2507_04786_b300/csrc/vcomm_reduce_inst.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


TRAFFIC_SOURCE = ("dram__bytes_read.sum + dram__bytes_write.sum per launch from a committed one-pass "
                  "ncu capture of the full-size launch (profiles/dram_traffic.txt), used only while "
                  "the kernel's sources are unchanged since; null otherwise")


def profiled_traffic(workload, proto):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    with open(p) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(x.split("=", 1) for x in line.split())
            if kv.get("workload") == workload and kv.get("proto") == proto and kv.get("src") == src:
                return float(kv["bytes_per_launch"])
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with `nvidia-smi -lms 100`
    (read only) while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._p = None

    def __enter__(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                        "--query-gpu=" + self.FIELDS,
                                        "--format=csv,noheader,nounits", "-lms", "100"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)     # first sample lands before the timed region starts
        except Exception:
            self._p = None
        return self

    def __exit__(self, *a):
        if self._p is None:
            return
        time.sleep(0.15)
        self._p.terminate()
        try:
            out, _ = self._p.communicate(timeout=5)
        except Exception:
            self._p.kill()
            out, _ = self._p.communicate()
        self.rows = [[x.strip() for x in l.split(",")] for l in out.splitlines() if l.strip()]

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[0]) for r in self.rows) if v is not None]
        mx = [v for v in (num(r[1]) for r in self.rows if len(r) > 1) if v is not None]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 2 + i and r[2 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg

def oracle_all_reduce(xs, dtype, op, nch, chunk, threads=1):
    """The CPU oracle's ring AllReduce of the whole buffers.  threads > 1:
    the same oracle function on every channel's slice, one host thread per
    slice (channels are independent and a slice run on one channel replays
    exactly that channel's loops, so the result is bit-identical; the oracle
    releases the interpreter lock while it runs)."""
    import oracle
    if threads <= 1:
        return oracle.all_reduce(xs, dtype, op, nch, chunk)
    from concurrent.futures import ThreadPoolExecutor
    n = xs[0].size
    es = oracle.ESIZE[dtype]
    outs = [np.empty_like(x) for x in xs]

    def one(ch):
        lo, ln = oracle.channel_range(n, es, nch, ch)
        if ln == 0:
            return
        part = oracle.all_reduce([x[lo:lo + ln] for x in xs], dtype, op, 1, chunk)
        for o, p_ in zip(outs, part):
            o[lo:lo + ln] = p_

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(nch)))
    return outs


def oracle_threads(nch):
    return max(1, min(os.cpu_count() or 1, nch))


def cpu_oracle_run(k, S_sample, proto, nch, chunk_steps, seed, reps=1, threads=1, xs=None):
    """Time the CPU oracle on a bounded sample of the workload (fp32 sum)."""
    import oracle
    n = S_sample // 4
    if xs is None:
        xs = inputs.workload(seed, k, n, "fp32", "normal")
    chunk = oracle.chunk_units(proto, 4, chunk_steps)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle_all_reduce(xs, "fp32", "sum", nch, chunk, threads)
        times.append(time.perf_counter() - t0)
    return times


def cpu_baseline(k, proto, nch, chunk_steps, seed):
    """The CPU oracle on the host cores, on a bounded sample: the headline
    AllReduce (k vranks, 37 channels) at 64 MiB per vrank, once with one
    thread per channel slice on all cores and once single-threaded (the same
    fold order, the same bits), plus the exactly-summable 4-vrank case
    (1,048,576 fp32 integers per vrank, Simple, one channel), reported as bus
    GB/s."""
    S = 64 << 20
    xs = inputs.workload(seed, k, S // 4, "fp32", "normal")
    thr = oracle_threads(nch)
    t_all = min(cpu_oracle_run(k, S, proto, nch, chunk_steps, seed, reps=2, threads=thr, xs=xs))
    t_one = cpu_oracle_run(k, S, proto, nch, chunk_steps, seed, reps=1, threads=1, xs=xs)[0]
    del xs
    import oracle
    e = workloads.EXACT
    n1 = e["count"]
    x1 = inputs.workload(e["seed"], e["nranks"], n1, "fp32", "int", lo=-1000, hi=1000)
    ch1 = oracle.chunk_units(e["proto"], 4, 1)
    t1 = []
    for _ in range(3):
        t0 = time.perf_counter()
        oracle.all_reduce(x1, "fp32", "sum", e["nchannels"], ch1)
        t1.append(time.perf_counter() - t0)
    t1 = min(t1)
    return {"value": round(busbw(S, k, t_all), 4), "unit": "GB/s", "cores": thr,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{k} vranks x {S >> 20} MiB fp32 ring AllReduce ({proto}, {nch} channels), "
                      f"one oracle thread per channel slice on {thr} of {os.cpu_count()} host "
                      f"cores, best of 2 runs ({t_all:.2f} s)",
            "single_thread": {"value": round(busbw(S, k, t_one), 4), "unit": "GB/s", "cores": 1,
                              "seconds": round(t_one, 3)},
            "exact_4vr_1Mi": {"workload": e["name"], "seconds": round(t1, 4), "cores": 1,
                              "algbw_GBps": round(n1 * 4 / t1 / 1e9, 4),
                              "busbw_GBps": round(busbw(n1 * 4, e["nranks"], t1), 4)}}


# ------------------------------------------------------------------ GPU leg

_HEADLINE_INPUTS = {}   # the headline's inputs, drawn once per process


def run_gpu(args, rank, world, proto=None, steps=None, e2e=True):
    import torch

    from paper_2507_04786_b300 import Comm

    w = workloads.HEADLINE
    k, S = w["nranks"], args.bytes
    n = S // 4
    proto = proto or args.proto
    steps = steps or args.steps
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    key = (w["seed"] + rank, k, n)
    if key not in _HEADLINE_INPUTS:
        _HEADLINE_INPUTS.clear()
        _HEADLINE_INPUTS[key] = inputs.workload(w["seed"] + rank, k, n, "fp32", w["dist"])
    xs = _HEADLINE_INPUTS[key]
    host = [torch.from_numpy(x).pin_memory() for x in xs]
    sends = [h.to(dev) for h in host]
    recvs = [torch.empty_like(s) for s in sends]
    comm = Comm(k, w["nchannels"])
    comm.set_plan(nchannels=w["nchannels"], chunk_steps=w["chunk_steps"])
    stream = torch.cuda.current_stream()

    def step():
        comm.all_reduce(sends, recvs, op="sum", algo="ring", proto=proto, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if comm.async_error() != "vSuccess":
        raise RuntimeError(comm.async_error())

    barrier(world)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        step()   # untimed: the GPU sat idle while the sampler started
        t0.record(stream)
        for i in range(steps):
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in evs]
    if comm.async_error() != "vSuccess":
        raise RuntimeError(comm.async_error())
    res = {"ms_per_step": total_ms / steps, "launch_ms": float(np.mean(launch_ms)),
           "clocks": clk.summary(), "launches": steps, "S": S, "k": k, "proto": proto}
    if not e2e:
        comm.destroy()
        return res

    # end to end: pinned host inputs -> device, AllReduce, results -> host.
    # Every step copies its own inputs in and its own result out inside the
    # timed region.  Two device buffer sets on three streams let the upload
    # of step i + 1 (one copy engine) run while step i's result comes back
    # (the other engine); a set is reused only after step i - 2 has read its
    # inputs and its result has left the device.
    e2e_steps = max(2, min(steps, 10))
    outs = [torch.empty_like(h).pin_memory() for h in host]
    sets = [(sends, recvs), ([torch.empty_like(x) for x in sends], [torch.empty_like(x) for x in sends])]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in, ev_red, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_event(e0)
    for i in range(e2e_steps):
        b = i % 2
        sb, rb = sets[b]
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_red[b])
            for h, x in zip(host, sb):
                x.copy_(h, non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if i >= 2:
            stream.wait_event(ev_out[b])
        comm.all_reduce(sb, rb, op="sum", algo="ring", proto=proto, stream=stream)
        ev_red[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_red[b])
            for o, r in zip(outs, rb):
                o.copy_(r, non_blocking=True)
            ev_out[b].record(s_out)
    stream.wait_stream(s_in)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if comm.async_error() != "vSuccess":
        raise RuntimeError(comm.async_error())
    want = [r.cpu() for r in sets[(e2e_steps - 1) % 2][1][:1]]
    if not torch.equal(outs[0].view(torch.int32), want[0].view(torch.int32)):
        raise RuntimeError("end-to-end result differs from the device result")
    comm.destroy()
    res["e2e_ms"] = e2e_ms
    return res


# ------------------------------------------------------------------ direct leg

def run_direct(args):
    """The headline workload (8 vranks x 256 MiB fp32, 37 channels) with the
    direct protocol: no FIFO, each unit's ring chain folded from the user
    buffers; 2kS algorithmic bytes.  Its output is compared bit for bit with
    a Simple call of the same plan."""
    import torch

    from paper_2507_04786_b300 import Comm
    w = workloads.HEADLINE
    k, S = w["nranks"], args.bytes
    n = S // 4
    xs = inputs.workload(w["seed"], k, n, "fp32", w["dist"])
    sends = [torch.from_numpy(x).cuda() for x in xs]
    del xs
    recvs = [torch.empty_like(t) for t in sends]
    comm = Comm(k, w["nchannels"])
    comm.set_plan(nchannels=w["nchannels"], chunk_steps=w["chunk_steps"])
    comm.all_reduce(sends, recvs, op="sum", algo="ring", proto="simple")
    ref = [r.clone() for r in recvs[:2]]
    for _ in range(args.warmup):
        comm.all_reduce(sends, recvs, op="sum", algo="ring", proto="direct")
    torch.cuda.synchronize()
    same = all(torch.equal(a.view(torch.int32), b.view(torch.int32)) for a, b in zip(ref, recvs[:2]))
    del ref
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    stream = torch.cuda.current_stream()
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        # untimed: the GPU sat idle while the sampler started
        comm.all_reduce(sends, recvs, op="sum", algo="ring", proto="direct", stream=stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            comm.all_reduce(sends, recvs, op="sum", algo="ring", proto="direct", stream=stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    err = comm.async_error()
    comm.destroy()
    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes(k, S, "direct")
    achieved = alg / (ms / 1e3) / 1e9
    return {"workload": w["name"], "proto": "direct", "ms_per_step": round(ms, 4),
            "busbw_GBps": round(busbw(S, k, ms / 1e3), 2),
            "algbw_GBps": round(S / (ms / 1e3) / 1e9, 2),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_launch": alg,
                         "peak_source": peak_kind,
                         "nominal_frac": round(achieved / NOMINAL_HBM_GBS, 4)},
            "equals_simple": bool(same), "clocks": clk.summary(), "status": err}


# ------------------------------------------------------------------ tile-engine group leg

def run_tile_group(args):
    """The headline workload (8 vranks x S fp32, direct protocol) as a group
    of two AllReduce calls on the two halves of every buffer: one launch of
    the tile engine (kBatchTiles: a producer warp issuing bulk copies, eight
    consumer warps folding from shared memory).  2kS algorithmic bytes; the
    output is compared bit for bit with one direct call on the whole
    buffers."""
    import torch

    from paper_2507_04786_b300 import Comm, group
    w = workloads.HEADLINE
    k, S = w["nranks"], args.bytes
    n = S // 4
    h = n // 2
    xs = inputs.workload(w["seed"], k, n, "fp32", w["dist"])
    sends = [torch.from_numpy(x).cuda() for x in xs]
    del xs
    recvs = [torch.empty_like(t) for t in sends]
    comm = Comm(k, w["nchannels"])
    stream = torch.cuda.current_stream()

    def grp():
        with group():
            comm.all_reduce([t[:h] for t in sends], [t[:h] for t in recvs], op="sum", algo="ring",
                            proto="direct", stream=stream)
            comm.all_reduce([t[h:] for t in sends], [t[h:] for t in recvs], op="sum", algo="ring",
                            proto="direct", stream=stream)

    grp()
    plans = comm.group_plans()
    torch.cuda.synchronize()
    got = [r.clone() for r in recvs[:2]]
    # the same halves as single calls (same plans): the group must give their bits
    for (lo, hi), p in zip(((0, h), (h, n)), plans):
        comm.set_plan(nchannels=p["nchannels"], chunk_steps=p["chunkSteps"])
        comm.all_reduce([t[lo:hi] for t in sends], [t[lo:hi] for t in recvs], op="sum", algo="ring",
                        proto="direct", stream=stream)
    torch.cuda.synchronize()
    same = all(torch.equal(a.view(torch.int32), b.view(torch.int32)) for a, b in zip(got, recvs[:2]))
    del got
    comm.clear_plan()
    for _ in range(args.warmup):
        grp()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        grp()   # untimed: the GPU sat idle while the sampler started
        for i in range(args.steps):
            evs[i][0].record(stream)
            grp()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    err = comm.async_error()
    comm.destroy()
    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes(k, S, "direct")
    achieved = alg / (ms / 1e3) / 1e9
    return {"workload": w["name"] + "-as-2-call-group", "proto": "direct", "kernel": "kBatchTiles",
            "ms_per_step": round(ms, 4), "busbw_GBps": round(busbw(S, k, ms / 1e3), 2),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_launch": alg,
                         "peak_source": peak_kind,
                         "nominal_frac": round(achieved / NOMINAL_HBM_GBS, 4)},
            "equals_single_calls": bool(same), "clocks": clk.summary(), "status": err}


# ------------------------------------------------------------------ all-to-all leg

def run_alltoall(args):
    """All-to-all (the grouped send / receive pattern) on 8 vranks, 256 MiB
    per vrank (blocks of 32 MiB), fp32: 2kS bytes (every block read once and
    written once)."""
    import torch

    from paper_2507_04786_b300 import Comm
    k, S = 8, args.bytes
    n = S // 4
    sends = [torch.randn(n, device="cuda") for _ in range(k)]
    recvs = [torch.empty_like(t) for t in sends]
    comm = Comm(k, 1)
    for _ in range(args.warmup):
        comm.all_to_all(sends, recvs)
    torch.cuda.synchronize()
    ok = all(torch.equal(recvs[j][r * (n // k):(r + 1) * (n // k)], sends[r][j * (n // k):(j + 1) * (n // k)])
             for r in (0, k - 1) for j in (0, 3, k - 1))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        evs[i][0].record()
        comm.all_to_all(sends, recvs)
        evs[i][1].record()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    err = comm.async_error()
    comm.destroy()
    peak, peak_kind = measured_peak()
    alg = 2 * k * S
    achieved = alg / (ms / 1e3) / 1e9
    return {"workload": f"alltoall-8vr-{S >> 20}MiB", "ms_per_step": round(ms, 4),
            "algbw_GBps": round(S / (ms / 1e3) / 1e9, 2),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "algorithmic_bytes_per_launch": alg,
                         "peak_source": peak_kind,
                         "nominal_frac": round(achieved / NOMINAL_HBM_GBS, 4)},
            "sampled_blocks_exact": bool(ok), "status": err}


# ------------------------------------------------------------------ batched leg

def run_batched(args):
    """64 AllReduce calls on 8 vranks, per-rank sizes log-uniform in
    4 KiB..64 MiB, dtypes fp32/bf16/int32, ops sum/max, plans from the
    autotuner: 64 plain calls per step vs one replay of the captured batch."""
    import torch

    from paper_2507_04786_b300 import Comm, group
    w = workloads.BATCHED
    k, nops = w["nranks"], w["nops"]
    g = np.random.default_rng(w["seed"])
    sizes = inputs.log_uniform_sizes(w["seed"], nops, w["lo_bytes"], w["hi_bytes"])
    tdt = {"fp32": torch.float32, "bf16": torch.bfloat16, "int32": torch.int32}
    ops = []
    for i in range(nops):
        dt = ("fp32", "bf16", "int32")[g.integers(3)]
        op = ("sum", "max")[g.integers(2)]
        es = 2 if dt == "bf16" else 4
        n = int(sizes[i]) // es
        s_ = [torch.ones(n, dtype=tdt[dt], device="cuda") for _ in range(k)]
        d_ = [torch.empty_like(t) for t in s_]
        ops.append((s_, d_, op, n * es))
    comm = Comm(k, w["nchannels"])
    t0 = time.time()
    comm.tune(colls=("allreduce",), max_bytes=w["hi_bytes"])
    tune_s = time.time() - t0
    comm.prepare(algos=("ring", "tree"), protos=("simple", "ll", "ll128"))
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()

    def plain():
        for s_, d_, op, _ in ops:
            comm.all_reduce(s_, d_, op=op, algo="auto", proto="auto", stream=stream)

    def batched():
        with group():
            for s_, d_, op, _ in ops:
                comm.all_reduce(s_, d_, op=op, algo="auto", proto="auto", stream=stream)

    steps = max(args.steps // 5, 5)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    plain_ms = timed(plain)
    with torch.cuda.stream(stream):
        batched()                               # fixes the plans before capture
    torch.cuda.synchronize()
    protos = [p["proto"] for p in comm.group_plans()]
    ndirect = sum(p == "direct" for p in protos)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batched()
    batch_ms = timed(graph.replay)
    err = comm.async_error()
    comm.destroy()
    total = sum(o[3] for o in ops)
    return {"workload": w["name"], "ops": nops, "nranks": k,
            "bytes_per_rank_total": total, "plain_ms": round(plain_ms, 4),
            "batched_graph_ms": round(batch_ms, 4), "speedup": round(plain_ms / batch_ms, 3),
            "plain_algbw_GBps": round(total / (plain_ms / 1e3) / 1e9, 2),
            "batched_algbw_GBps": round(total / (batch_ms / 1e3) / 1e9, 2),
            "direct_calls": ndirect, "fifo_calls": len(protos) - ndirect,
            # the group's kernels: one tile-engine launch for its direct calls,
            # one batch kernel for its FIFO calls
            "graph_launches": int(ndirect > 0) + int(len(protos) > ndirect),
            "tune_seconds": round(tune_s, 1), "status": err}


# ------------------------------------------------------------------ small-message leg

def run_small(args):
    """Latency of small collectives (the flag round-trip bound regime):
    each collective at 1 KiB and 64 KiB per rank on 8 and 16 vranks, with the
    library's Auto plan and with the paper's LL / LL128 protocols forced (at
    their best channel count).  Device time per call: a CUDA graph of 10
    calls, median of 21 replays."""
    import torch

    from paper_2507_04786_b300 import Comm
    w = workloads.SMALL
    reps_in_graph, replays = 10, 21

    def call(c, coll, a, b, proto, s):
        algo = "auto" if (coll == "allreduce" and proto == "auto") else (
            "tree" if coll == "allreduce" else "ring")
        if coll == "allreduce":
            c.all_reduce(a, b, algo=algo, proto=proto, stream=s)
        elif coll == "reducescatter":
            c.reduce_scatter(a, b, algo="ring", proto=proto, stream=s)
        elif coll == "allgather":
            c.all_gather(a, b, algo="ring", proto=proto, stream=s)
        elif coll == "broadcast":
            c.broadcast(a, b, root=0, algo="ring", proto=proto, stream=s)
        else:
            c.reduce(a, b, root=0, algo="ring", proto=proto, stream=s)

    def graph_us(c, coll, a, b, proto):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            for _ in range(3):
                call(c, coll, a, b, proto, stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(reps_in_graph):
                call(c, coll, a, b, proto, stream)
        g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(replays):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3 / reps_in_graph)
        return round(float(np.median(ts)), 2)

    rows = []
    for k in w["nranks"]:
        big = [torch.randn(max(w["bytes"]) // 4, device="cuda") for _ in range(k)]
        out = [torch.empty_like(x) for x in big]
        c = Comm(k, w["nchannels"])
        c.prepare(algos=("ring", "tree"), protos=("ll", "ll128"))
        for coll in w["colls"]:
            for S in w["bytes"]:
                n = S // 4
                if coll == "reducescatter":
                    a, b = [x[:n] for x in big], [y[:n // k] for y in out]
                elif coll == "allgather":
                    a, b = [x[:n // k] for x in big], [y[:n] for y in out]
                else:
                    a, b = [x[:n] for x in big], [y[:n] for y in out]
                row = {"coll": coll, "nranks": k, "bytes_per_rank": S}
                c.clear_plan()
                row["us_auto"] = graph_us(c, coll, a, b, "auto")
                p = c.last_plan()
                row["plan"] = f"{p['algo']}/{p['proto']}/{p['nchannels']}ch"
                for proto in ("ll", "ll128"):          # the paper's protocols, best channels
                    best = None
                    for C in w["ll_channels"]:
                        c.set_plan(nchannels=C, chunk_steps=1)
                        t = graph_us(c, coll, a, b, proto)
                        if best is None or t < best[0]:
                            best = (t, C)
                    row["us_" + proto], row[proto + "_channels"] = best
                c.clear_plan()
                rows.append(row)
        err = c.async_error()
        c.destroy()
        if err != "vSuccess":
            return {"workload": w["name"], "status": err}
    return {"workload": w["name"], "timing": "CUDA graph of 10 calls, median of 21 replays",
            "rows": rows, "status": "vSuccess"}


# ------------------------------------------------------------------ served leg

def fifo_proto(nbytes):
    """The paper's protocol choice by size (Sec. III-D: LL for small, LL128 for
    medium, Simple for large messages)."""
    return "ll" if nbytes < (64 << 10) else ("ll128" if nbytes < (2 << 20) else "simple")


SERVE_NAMES = {"streams": "continuous_batching_streams", "batch": "continuous_batching",
               "plain": "per_call", "tiles": "continuous_batching_tiles"}


def served_requests(nreq, seed=None):
    """The served workload's request stream: (collective, dtype, vranks,
    count, per-rank bytes S) per request and the Poisson arrival times."""
    w = workloads.SERVED
    seed = w["seed"] if seed is None else seed
    g = np.random.default_rng(seed)
    gaps = g.exponential(1.0 / w["rate_per_s"], nreq)
    arrivals = np.cumsum(gaps)
    sizes = inputs.log_uniform_sizes(seed, nreq, w["lo_bytes"], w["hi_bytes"])
    colls = g.integers(0, 3, nreq)
    ks = g.integers(2, w["max_ranks"] + 1, nreq)
    dts = g.integers(0, 2, nreq)
    names = ("allreduce", "reducescatter", "allgather")
    reqs = []
    for i in range(nreq):
        dt = ("fp32", "bf16")[dts[i]]
        es = 4 if dt == "fp32" else 2
        k = int(ks[i])
        coll = names[colls[i]]
        n = max(16 // es, int(sizes[i]) // es)            # S = the larger per-rank buffer
        if coll != "allreduce":
            n = max(1, n // k)
        reqs.append((coll, dt, k, n, int(sizes[i])))
    return reqs, arrivals


def served_pool():
    """Resident inputs: every request reads the same buffers (one per vrank
    and dtype, the largest request's size)."""
    import torch
    w = workloads.SERVED
    hi = w["hi_bytes"]
    pool = {"fp32": [torch.ones(hi // 4, dtype=torch.float32, device="cuda") for _ in range(w["max_ranks"])],
            "bf16": [torch.ones(hi // 2, dtype=torch.bfloat16, device="cuda") for _ in range(w["max_ranks"])]}
    torch.cuda.synchronize()
    return pool


def user_bytes(coll, k, S):
    """HBM bytes a request must move without a FIFO: AllReduce 2kS, ReduceScatter
    and AllGather (k + 1) S."""
    return 2 * k * S if coll == "allreduce" else (k + 1) * S


def run_saturation(args, modes=("plain", "tiles"), nreq=None, outstanding=None, repeats=3):
    """Closed loop: the served workload's requests with `outstanding` of them
    in flight at all times (a new one is submitted as soon as one completes),
    default protocol; the largest request rate and HBM rate each mode
    sustains, with the latency it costs.  The modes alternate over `repeats`
    runs (a closed loop's rates swing from run to run); each figure is the
    median over the runs, the per-run values beside it."""
    from paper_2507_04786_b300 import Server
    w = workloads.SERVED
    nreq = nreq or w["saturation_requests"]
    outstanding = outstanding or w["saturation_outstanding"]
    reqs, _ = served_requests(nreq)
    pool = served_pool()
    res = {"workload": w["name"].replace("poisson-2000rps", "closed-loop"), "requests": nreq,
           "outstanding": outstanding, "protocol": "auto (direct)", "repeats": repeats}
    runs = {m: [] for m in modes}
    for _ in range(repeats):
        for mode in modes:
            srv = Server(mode=mode, max_ranks=w["max_ranks"], mem_budget=w["budget_bytes"],
                         small_gangs=w["small_lanes"] if mode == "streams" else 1)
            live = {}
            lats = []
            nxt = 0
            t0 = time.monotonic_ns()
            while nxt < min(outstanding, nreq):
                coll, dt, k, n, S = reqs[nxt]
                live[srv.submit(coll, pool[dt][:k], n, dt, "sum", proto="auto", release=True)] = nxt
                nxt += 1
            deadline = time.time() + 120
            while live and time.time() < deadline:
                for t in list(live):
                    state, lat, _, _ = srv.query(t)
                    if state in ("done", "failed"):
                        lats.append(lat / 1e6)
                        srv.release(t)
                        del live[t]
                        if nxt < nreq:
                            coll, dt, k, n, S = reqs[nxt]
                            live[srv.submit(coll, pool[dt][:k], n, dt, "sum", proto="auto", release=True)] = nxt
                            nxt += 1
            span = (time.monotonic_ns() - t0) / 1e9
            st = srv.stats()
            srv.destroy()
            lats = np.array(lats)
            total = sum(user_bytes(c, k, S) for c, _, k, _, S in reqs[:len(lats)])
            runs[mode].append({"requests_per_s": len(lats) / span, "hbm_GBps": total / span / 1e9,
                               "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
                               "completed": int(st["completed"]), "failed": int(st["failed"])})
    for mode in modes:
        rs = runs[mode]
        out = {}
        for key, nd in (("requests_per_s", 1), ("hbm_GBps", 1), ("p50_ms", 4), ("p99_ms", 4)):
            vals = [r[key] for r in rs]
            out[key] = round(float(np.median(vals)), nd)
            out[key + "_runs"] = [round(v, nd) for v in vals]
        out["completed"] = sum(r["completed"] for r in rs)
        out["failed"] = sum(r["failed"] for r in rs)
        res[SERVE_NAMES[mode]] = out
    del pool
    return res


def run_served(args, rate=None, nreq=None, modes=("batch", "plain"), protocol="fifo"):
    """Poisson arrivals (mean 2000/s) of AllReduce / AllGather / ReduceScatter
    requests on 2..16 vranks, per-rank sizes log-uniform in 1 KiB..128 MiB,
    fp32/bf16, admitted under a 40 GB budget, the same request stream served by
    continuous batching on resident gangs and by one launch per request on one
    stream (and, for `modes` with "streams", continuous batching on lanes of
    streams); `protocol` "fifo": the paper's protocols by size, "auto": the
    library's choice (the direct protocol)."""
    import torch

    from paper_2507_04786_b300 import Server
    w = workloads.SERVED
    nreq = nreq or args.serve_requests
    rate = rate or w["rate_per_s"]
    reqs, arrivals = served_requests(nreq)
    if rate != w["rate_per_s"]:
        arrivals = arrivals * (w["rate_per_s"] / rate)
    pool = served_pool()
    out = {}
    for mode in modes:
        srv = Server(mode=mode, max_ranks=w["max_ranks"], mem_budget=w["budget_bytes"],
                     small_gangs=w["small_lanes"] if mode == "streams" else 1)
        tickets = []
        t0 = time.monotonic_ns() + 20_000_000
        for i, (coll, dt, k, n, S) in enumerate(reqs):
            due = t0 + int(arrivals[i] * 1e9)
            while time.monotonic_ns() < due:
                pass
            proto = fifo_proto(S) if protocol == "fifo" else "auto"
            tickets.append(srv.submit(coll, pool[dt][:k], n, dt, "sum", proto=proto, release=True,
                                      arrival_ns=due))
        deadline = time.time() + 120
        while srv.stats()["completed"] + srv.stats()["failed"] < nreq and time.time() < deadline:
            time.sleep(0.005)
        st = srv.stats()
        lats, ends, svc_big, svc_small = [], [], [], []
        for i, t in enumerate(tickets):
            state, lat, _, _ = srv.query(t)
            if state == "done":
                lats.append(lat / 1e6)
                ends.append(arrivals[i] + lat / 1e9)
                if srv.last_service_ns > 0:
                    (svc_big if reqs[i][4] >= (4 << 20) else svc_small).append(srv.last_service_ns / 1e6)
            srv.release(t)
        srv.destroy()
        lats = np.array(lats, dtype=np.float64)
        span = (max(ends) - arrivals[0]) if ends else float("nan")
        total = sum(r[4] * r[2] for r in reqs)
        out[mode] = {"p50_ms": round(float(np.percentile(lats, 50)), 4) if lats.size else None,
                     "p99_ms": round(float(np.percentile(lats, 99)), 4) if lats.size else None,
                     "mean_ms": round(float(lats.mean()), 4) if lats.size else None,
                     "completed": int(st["completed"]), "failed": int(st["failed"]),
                     "requests_per_s": round(len(lats) / span, 1),
                     "GBps": round(total / span / 1e9, 2),
                     "max_inflight_GB": round(st["maxInflightBytes"] / 1e9, 2),
                     "mean_service_ms_large": round(float(np.mean(svc_big)), 4) if svc_big else None,
                     "mean_service_ms_small": round(float(np.mean(svc_small)), 4) if svc_small else None}
    del pool
    names = SERVE_NAMES
    res = {"workload": w["name"] if rate == w["rate_per_s"] else f"served-poisson-{int(rate)}rps",
           "requests": nreq, "rate_per_s": rate, "budget_GB": w["budget_bytes"] / 1e9,
           "protocol": ("the paper's FIFO protocols by size (LL < 64 KiB <= LL128 < 2 MiB <= Simple)"
                        if protocol == "fifo" else "auto (direct)"),
           "latency": "completion seen by the host minus the scheduled arrival (queueing included)"}
    for m in modes:
        res[names[m]] = out[m]
    return res


# ------------------------------------------------------------------ protocol sweep

def run_sweep(path, protos=("simple", "ll", "ll128", "cluster"), algo="ring"):
    """AllReduce on 8 vranks (ring, or the double binary tree): per-rank sizes 1 KiB..256 MiB (powers of
    4) x fp32 / bf16 x the given protocols (default Simple / LL / LL128 and
    the cluster protocol up to 4 MiB) x 1 / 4 / 16 / 32 channels, N(0,1)
    values; one JSON line per point (median of timed launches)."""
    import torch

    from paper_2507_04786_b300 import Comm, VcommError
    k = 8
    top = max(workloads.SWEEP_BYTES)
    base = {dt: [torch.randn(top // es, device="cuda").to(t) for _ in range(k)]
            for dt, es, t in (("fp32", 4, torch.float32), ("bf16", 2, torch.bfloat16))}
    outs = {dt: [torch.empty_like(x) for x in xs] for dt, xs in base.items()}
    comm = Comm(k, max(workloads.SWEEP_CHANNELS))
    rows = []
    with open(path, "w") as f:
        for dt in ("fp32", "bf16"):
            es = 4 if dt == "fp32" else 2
            for S in workloads.SWEEP_BYTES:
                n = S // es
                xs = [x[:n] for x in base[dt]]
                ys = [y[:n] for y in outs[dt]]
                for proto in protos:
                    if proto == "cluster" and S > workloads.SWEEP_CLUSTER_MAX:
                        continue
                    for C in workloads.SWEEP_CHANNELS:
                        comm.set_plan(nchannels=C, chunk_steps=1)
                        try:
                            for _ in range(2):
                                comm.all_reduce(xs, ys, algo=algo, proto=proto)
                        except VcommError as e:      # e.g. more CTAs than can be co-resident
                            f.write(json.dumps({"dtype": dt, "bytes_per_rank": S, "algo": algo, "proto": proto,
                                                "nchannels": C, "refused": e.name}) + "\n")
                            continue
                        torch.cuda.synchronize()
                        reps = 5 if S >= (16 << 20) else 20
                        ts = []
                        for _ in range(reps):
                            e0 = torch.cuda.Event(enable_timing=True)
                            e1 = torch.cuda.Event(enable_timing=True)
                            e0.record()
                            comm.all_reduce(xs, ys, algo=algo, proto=proto)
                            e1.record()
                            e1.synchronize()
                            ts.append(e0.elapsed_time(e1))
                        ms = float(np.median(ts))
                        alg = algorithmic_bytes(k, S, proto)
                        row = {"dtype": dt, "bytes_per_rank": S, "algo": algo, "proto": proto, "nchannels": C,
                               "us": round(ms * 1e3, 2), "busbw_GBps": round(busbw(S, k, ms / 1e3), 2),
                               "hbm_frac": round(alg / (ms / 1e3) / 1e9 / measured_peak()[0], 4)}
                        rows.append(row)
                        f.write(json.dumps(row) + "\n")
    assert comm.async_error() == "vSuccess"
    comm.destroy()
    # best per (dtype, size)
    best = {}
    for r in rows:
        key = (r["dtype"], r["bytes_per_rank"])
        if key not in best or r["us"] < best[key]["us"]:
            best[key] = r
    return [best[k_] for k_ in sorted(best)]


def run_hop(args):
    """Per-hop latency of the FIFO protocols (vDebugHopLatency): rings of 8
    and 16 CTAs on consecutive SM ids, on SM ids alternating between the two
    halves of the id range, and as one thread-block cluster; and an LL
    ping-pong between SM 0 and every other SM (the spread shows whether some
    pairs pay more, e.g. across the two dies)."""
    import torch

    from paper_2507_04786_b300 import VcommError
    from paper_2507_04786_b300.binding import debug_hop_latency
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    half = nsm // 2
    rows = []
    for proto in ("ll", "ll128", "simple"):
        for k in (8, 16):
            rings = {"consecutive": list(range(k)),
                     "alternating_halves": [i // 2 + (i % 2) * half for i in range(k)],
                     "cluster": None}
            for name, sms in rings.items():
                try:
                    ns, got = debug_hop_latency(proto, sms, n=k, laps=2000)
                    rows.append({"proto": proto, "ring": name, "ctas": k, "us_per_hop": round(ns / 1e3, 3),
                                 "sms": got})
                except VcommError as e:
                    rows.append({"proto": proto, "ring": name, "ctas": k, "error": e.name})
    pp = {}
    for j in range(1, nsm):
        try:
            ns, _ = debug_hop_latency("ll", [0, j], laps=500)
            pp[j] = round(ns / 1e3, 3)
        except VcommError as e:
            pp[j] = e.name
    vals = np.array([v for v in pp.values() if isinstance(v, float)])
    summary = {}
    if vals.size:
        lo = float(vals.min())
        summary = {"min_us": lo, "median_us": float(np.median(vals)), "max_us": float(vals.max()),
                   "sms_above_1.5x_min": int((vals > 1.5 * lo).sum()), "sms": int(vals.size)}
    return {"paper_us_per_hop": {"simple": 6, "ll": 1, "ll128": 2}, "rings": rows,
            "pingpong_ll_from_sm0": summary, "pingpong_ll_us_by_sm": pp}


COLL_SWEEP_BYTES = [workloads.KiB * 4 ** i for i in range(1, 9)] + [128 << 20]


def coll_bytes(coll, k, S, proto):
    """System-wide algorithmic bytes of one collective, S = the larger
    per-rank buffer (ReduceScatter sendbuf, AllGather recvbuf): user bytes
    plus 2(k-1)S x f of FIFO writes and reads (f = 0 without a FIFO)."""
    f = FIFO_FACTOR[proto]
    user = {"allreduce": 2 * k * S, "reducescatter": k * S + S, "allgather": S + k * S,
            "broadcast": S + k * S, "reduce": k * S + S}[coll]
    return user + (4 if coll == "allreduce" else 2) * (k - 1) * S * f


def run_coll_sweep(path, protos=("direct", "simple"), nchannels=16):
    """ReduceScatter, AllGather, Broadcast (root 0) and Reduce (root 0) on 8
    and 16 vranks, fp16 and int32 (sum), per-rank sizes 4 KiB..64 MiB
    (powers of 4) and 128 MiB, ring, the given protocols at `nchannels`
    channels; one JSON line per point (median of launches timed alone)."""
    import torch

    from paper_2507_04786_b300 import Comm
    top = max(COLL_SWEEP_BYTES)
    rows = []
    with open(path, "w") as f:
        for k in (8, 16):
            comm = Comm(k, nchannels)
            comm.set_plan(nchannels=nchannels, chunk_steps=1)
            for dt, t in (("fp16", torch.float16), ("int32", torch.int32)):
                es = torch.tensor([], dtype=t).element_size()
                big = [torch.ones(top // es, device="cuda", dtype=t) for _ in range(k)]
                out = [torch.empty(top // es, device="cuda", dtype=t) for _ in range(k)]
                for S in COLL_SWEEP_BYTES:
                    n = S // es
                    xs, ys = [x[:n] for x in big], [y[:n] for y in out]
                    blk = [y[:n // k] for y in out]
                    for coll in ("reducescatter", "allgather", "broadcast", "reduce"):
                        for proto in protos:
                            if coll == "reducescatter":
                                call = lambda: comm.reduce_scatter(xs, blk, algo="ring", proto=proto)
                            elif coll == "allgather":
                                call = lambda: comm.all_gather([x[:n // k] for x in xs], ys, algo="ring",
                                                               proto=proto)
                            elif coll == "broadcast":
                                call = lambda: comm.broadcast(xs, ys, root=0, algo="ring", proto=proto)
                            else:
                                call = lambda: comm.reduce(xs, [ys[0]] + [None] * (k - 1), root=0,
                                                           algo="ring", proto=proto)
                            for _ in range(2):
                                call()
                            torch.cuda.synchronize()
                            ts = []
                            for _ in range(5 if S >= (16 << 20) else 20):
                                e0 = torch.cuda.Event(enable_timing=True)
                                e1 = torch.cuda.Event(enable_timing=True)
                                e0.record()
                                call()
                                e1.record()
                                e1.synchronize()
                                ts.append(e0.elapsed_time(e1))
                            ms = float(np.median(ts))
                            alg = coll_bytes(coll, k, S, proto)
                            row = {"coll": coll, "nranks": k, "dtype": dt, "bytes_per_rank": S, "proto": proto,
                                   "nchannels": nchannels, "us": round(ms * 1e3, 2),
                                   "hbm_frac": round(alg / (ms / 1e3) / 1e9 / measured_peak()[0], 4)}
                            rows.append(row)
                            f.write(json.dumps(row) + "\n")
                del big, out
            assert comm.async_error() == "vSuccess"
            comm.destroy()
    return rows


def headline_leg(args, rank, world, proto, wname):
    """The headline workload with another FIFO protocol (same channels, same
    chunk), timed the same way on the launching stream: its own roofline
    against the bytes that protocol must move."""
    r = run_gpu(args, rank, world, proto=proto, steps=max(5, args.steps // 2), e2e=False)
    ms = reduce_max(world, r["ms_per_step"])
    launch_ms = reduce_max(world, r["launch_ms"])
    k, S = r["k"], r["S"]
    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes(k, S, proto)
    achieved = alg / (launch_ms / 1e3) / 1e9
    return {"proto": proto, "value": round(job_value(world, S, k, ms), 3), "unit": "GB/s",
            "ms_per_step": round(ms, 4), "steps": r["launches"],
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": profiled_traffic(wname, proto), "traffic_source": TRAFFIC_SOURCE,
                         "algorithmic_bytes_per_launch": alg, "peak_source": peak_kind,
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "nominal_frac": round(achieved / NOMINAL_HBM_GBS, 4)},
            "clocks": r["clocks"]}


def run_chain_sweep(path):
    """Ring Broadcast (root 0), Reduce (root 0) and AllReduce with the Simple
    protocol, fp16, 128 MiB per vrank, on 8, 12 and 16 vranks at pinned
    channel counts on both sides of SMs / vranks (the chains' channels are
    capped there; the plan read back shows the channels that ran); median of
    5 launches timed alone.  One JSON line per point."""
    import torch

    from paper_2507_04786_b300 import Comm
    S = 128 << 20
    rows = []
    with open(path, "w") as f:
        for k, chans in ((8, (8, 16, 18)), (12, (8, 12, 16)), (16, (4, 8, 9, 10, 12, 16))):
            n = S // 2
            xs = [torch.ones(n, dtype=torch.float16, device="cuda") for _ in range(k)]
            ys = [torch.empty_like(x) for x in xs]
            c = Comm(k, max(chans))
            for C in chans:
                c.set_plan(nchannels=C, chunk_steps=1)
                for coll in ("broadcast", "reduce", "allreduce"):
                    if coll == "broadcast":
                        call = lambda: c.broadcast(xs, ys, root=0, algo="ring", proto="simple")
                    elif coll == "reduce":
                        call = lambda: c.reduce(xs, [ys[0]] + [None] * (k - 1), root=0, algo="ring",
                                                proto="simple")
                    else:
                        call = lambda: c.all_reduce(xs, ys, algo="ring", proto="simple")
                    for _ in range(2):
                        call()
                    torch.cuda.synchronize()
                    ts = []
                    for _ in range(5):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        call()
                        e1.record()
                        e1.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    row = {"coll": coll, "nranks": k, "pinned_channels": C,
                           "channels": c.last_plan()["nchannels"], "ms": round(float(np.median(ts)), 3)}
                    rows.append(row)
                    f.write(json.dumps(row) + "\n")
            assert c.async_error() == "vSuccess"
            c.destroy()
            del xs, ys
    return rows


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, x):
    """The slowest replica's value (the job's time is the max over ranks)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, S, k, max_ms):
    """Whole-job bus bandwidth: every replica moved S per vrank; the job took
    the slowest replica's time."""
    return world * busbw(S, k, max_ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--proto", default="simple", choices=["simple", "ll", "ll128", "direct"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-ll128", action="store_true",
                    help="skip the LL128 leg of the headline workload")
    ap.add_argument("--serve-requests", type=int, default=workloads.SERVED["bench_requests"],
                    help="requests of the served legs of the other modes and the paper's protocols")
    ap.add_argument("--serve-requests-direct", type=int, default=workloads.SERVED["requests"],
                    help="requests of the default-protocol served comparison (the whole stream)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--extras", default="direct,tilegroup,alltoall,small,batched,served,saturation,hop",
                    help="the extra legs to run, comma separated (profiling captures run one)")
    ap.add_argument("--sweep", default=None,
                    help="run the protocol x size x channel sweep, write JSON lines here, exit")
    ap.add_argument("--sweep-protos", default="simple,ll,ll128,cluster",
                    help="protocols of the sweep, comma separated (direct too)")
    ap.add_argument("--sweep-algo", default="ring", choices=["ring", "tree"],
                    help="algorithm of the sweep")
    ap.add_argument("--sweep-colls", default=None,
                    help="sweep ReduceScatter / AllGather / Broadcast / Reduce (direct and Simple), "
                         "write JSON lines here, exit")
    ap.add_argument("--sweep-chains", default=None,
                    help="time ring Broadcast / Reduce / AllReduce (Simple, fp16, 128 MiB) over vranks and "
                         "channels, write JSON lines here, exit")
    ap.add_argument("--bytes", type=int, default=workloads.HEADLINE["bytes_per_rank"],
                    help="bytes per vrank (default: the headline's 256 MiB; smaller sizes are "
                         "for profiling captures only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.sweep:
        for r in run_sweep(args.sweep, tuple(args.sweep_protos.split(",")), args.sweep_algo):
            print(json.dumps(r))
        return
    if args.sweep_colls:
        run_coll_sweep(args.sweep_colls)
        return
    if args.sweep_chains:
        for r in run_chain_sweep(args.sweep_chains):
            print(json.dumps(r))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")

    w = workloads.HEADLINE
    k, S = w["nranks"], args.bytes
    wname = w["name"] if S == w["bytes_per_rank"] else f"ring-allreduce-8vr-{S >> 20}MiB"
    config = {"workload": wname, "nranks": k, "bytes_per_rank": S, "dtype": "fp32",
              "op": "sum", "algo": "ring", "proto": args.proto, "nchannels": w["nchannels"],
              "chunk_steps": w["chunk_steps"], "values": "N(0,1)",
              "l2": f"inputs {k * S >> 20} MiB and outputs {k * S >> 20} MiB per step vs the "
                    f"126 MB L2 (no flush)",
              "replicas": world}
    metric = "8-vrank ring AllReduce bus bandwidth"

    if args.impl == "reference":
        if rank != 0:
            return
        reps = max(1, args.warmup) + args.steps
        # bounded sample: 8 MiB per vrank, one oracle AllReduce per step, one
        # oracle thread per channel slice on the host cores
        S_s = 8 << 20
        thr = oracle_threads(w["nchannels"])
        times = cpu_oracle_run(k, S_s, args.proto, w["nchannels"], w["chunk_steps"], w["seed"],
                               reps=reps, threads=thr)[args.warmup:]
        t = float(np.mean(times))
        v = busbw(S_s, k, t)
        line = {"metric": metric, "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "impl": "reference", "config": config,
                "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": thr,
                                 "host_cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"{k} vranks x {S_s >> 20} MiB per step, CPU oracle with "
                                           f"one thread per channel slice on {thr} host cores"},
                "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    r = run_gpu(args, rank, world)
    ms = reduce_max(world, r["ms_per_step"])
    launch_ms = reduce_max(world, r["launch_ms"])
    e2e_ms = reduce_max(world, r["e2e_ms"])
    if rank != 0:
        return
    value = job_value(world, S, k, ms)
    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes(k, S, args.proto)
    achieved = alg / (launch_ms / 1e3) / 1e9
    line = {
        "metric": metric, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config,
        "algbw_GBps": round(S / (ms / 1e3) / 1e9, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": profiled_traffic(wname, args.proto),
                     "traffic_source": TRAFFIC_SOURCE,
                     "algorithmic_bytes_per_launch": alg, "peak_source": peak_kind,
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "nominal_frac": round(achieved / NOMINAL_HBM_GBS, 4)},
        "e2e": {"value": round(world * busbw(S, k, e2e_ms / 1e3), 3), "unit": "GB/s",
                "h2d_bytes_per_step": k * S, "d2h_bytes_per_step": k * S},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    if args.proto == "simple" and not args.no_ll128:
        line["ll128"] = headline_leg(args, rank, world, "ll128", wname)
    legs = set(args.extras.split(","))
    if not args.no_extras and world == 1:
        if "direct" in legs:
            line["direct"] = run_direct(args)
        if "tilegroup" in legs:
            line["tile_group"] = run_tile_group(args)
        if "alltoall" in legs:
            line["alltoall"] = run_alltoall(args)
        if "small" in legs:
            line["small_messages"] = run_small(args)
        if "batched" in legs:
            line["batched"] = run_batched(args)
        if "served" in legs:
            # the default protocol over the whole stream: one launch per
            # request against continuous batching of tiles; the other modes
            # and the paper's protocols on the first 20,000 requests
            line["served_direct"] = run_served(args, nreq=args.serve_requests_direct,
                                               modes=("plain", "tiles"), protocol="auto")
            line["served_direct_other_modes"] = run_served(args, modes=("streams", "batch"), protocol="auto")
            line["served"] = run_served(args)
        if "saturation" in legs:
            line["saturation"] = run_saturation(args)
        if "hop" in legs:
            line["hop_latency"] = run_hop(args)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(k, args.proto, w["nchannels"], w["chunk_steps"],
                                            w["seed"])
    print(json.dumps(line))


if __name__ == "__main__":
    main()
