"""Named workloads: the shapes the benchmark times and the tests check.

Each workload is a plain dict; sizes are per vrank.  The headline is an
8-vrank ring AllReduce of 256 MiB per vrank (fp32 sum, N(0, 1) values),
timed with the Simple and LL128 protocols.
"""
MiB = 1 << 20
KiB = 1 << 10

HEADLINE = {
    "name": "ring-allreduce-8vr-256MiB",
    "coll": "allreduce",
    "algo": "ring",
    "nranks": 8,
    "bytes_per_rank": 256 * MiB,
    "dtype": "fp32",
    "op": "sum",
    "dist": "normal",
    "seed": 1,
    "protos": ("simple", "ll128"),
    "nchannels": 37,          # 8 x 37 = 296 CTAs: two per SM on 148 SMs
    "chunk_steps": 1,
}

# the exactly-summable correctness case: 4 vranks, 1,048,576 fp32 integers
# uniform in [-1000, 1000], Simple, one channel, seed 0
EXACT = {
    "name": "ring-allreduce-4vr-1Mi-int-fp32",
    "nranks": 4,
    "count": 1 << 20,
    "dtype": "fp32",
    "proto": "simple",
    "nchannels": 1,
    "seed": 0,
}

# 64 concurrent AllReduce calls in one persistent launch (group + CUDA graph)
BATCHED = {
    "name": "batched-64-allreduce-8vr-4KiB-64MiB",
    "nranks": 8,
    "nops": 64,
    "lo_bytes": 4 * KiB,
    "hi_bytes": 64 * MiB,
    "nchannels": 37,
    "seed": 3,
}

# Poisson stream of AllReduce / ReduceScatter / AllGather requests
SERVED = {
    "name": "served-poisson-2000rps-2to16vr-1KiB-128MiB",
    "rate_per_s": 2000.0,
    "max_ranks": 16,
    "lo_bytes": 1 * KiB,
    "hi_bytes": 128 * MiB,
    "budget_bytes": 40 * 10 ** 9,
    "requests": 100_000,          # the default-protocol comparison runs all of them
    "bench_requests": 20_000,     # the other served legs: 10 s of arrivals per mode
    "saturation_requests": 8_000,        # closed loop: requests per mode
    "saturation_outstanding": 32,        # closed loop: requests kept in flight
    "small_lanes": 4,             # continuous batching on streams: lanes for small requests
    "seed": 4,
}

# per-rank message sizes of the protocol sweep: 1 KiB .. 256 MiB in powers of 4
SWEEP_BYTES = [KiB * 4 ** i for i in range(10)]
SWEEP_CHANNELS = (1, 4, 16, 32)
SWEEP_CLUSTER_MAX = 4 * MiB   # the cluster protocol is swept up to 4 MiB per rank

# small-message latency: every collective at 1 KiB and 64 KiB per rank on 8
# and 16 vranks, fp32 N(0,1) (the per-hop latency regime)
SMALL = {
    "name": "small-messages-8and16vr-1KiB-64KiB",
    "nranks": (8, 16),
    "bytes": (1 * KiB, 64 * KiB),
    "colls": ("allreduce", "reducescatter", "allgather", "broadcast", "reduce"),
    "nchannels": 8,
    "ll_channels": (1, 2, 4, 8),   # LL / LL128 are timed at each; the best is kept
}
