"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws numbers; it holds none of the collectives' arithmetic.
Every vrank r of a workload seeded `seed` draws from its own PCG64 stream
(SeedSequence([seed, r])), so the inputs of one rank never depend on the
number of ranks.  Floating-point values are drawn in fp64 and converted to the
target dtype by numpy (fp32, fp16) or torch (bf16); bf16 arrays are returned as
uint16 bit patterns, fp16 as numpy float16.

Distributions follow the workloads the collectives are measured on: N(0, 1)
for the protocol sweep, uniform [-1, 1] for fp16, integers uniform in an
inclusive range for int32 and for the exactly-summable fp32 case.
"""
from __future__ import annotations

import math

import numpy as np

NP_DTYPE = {"int32": np.int32, "fp32": np.float32, "fp16": np.float16, "bf16": np.uint16,
            "int8": np.int8, "uint8": np.uint8, "uint32": np.uint32, "int64": np.int64,
            "uint64": np.uint64, "fp64": np.float64}
ESIZE = {"int32": 4, "fp32": 4, "fp16": 2, "bf16": 2, "int8": 1, "uint8": 1, "uint32": 4,
         "int64": 8, "uint64": 8, "fp64": 8}
INT_TYPES = ("int8", "uint8", "int32", "uint32", "int64", "uint64")


def rng_for(seed: int, rank: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, rank])))


def _to_bf16_bits(x64: np.ndarray) -> np.ndarray:
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x64, dtype=np.float64)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy()


def cast(x64: np.ndarray, dtype: str) -> np.ndarray:
    if dtype == "fp32":
        return x64.astype(np.float32)
    if dtype == "fp16":
        return x64.astype(np.float16)
    if dtype == "bf16":
        return _to_bf16_bits(x64)
    if dtype == "fp64":
        return np.asarray(x64, dtype=np.float64).copy()
    if dtype in INT_TYPES:
        return x64.astype(NP_DTYPE[dtype])
    raise ValueError(dtype)


def rank_values(seed: int, rank: int, n: int, dtype: str, dist: str = "normal",
                lo: int = -1000, hi: int = 1000) -> np.ndarray:
    """n values of one vrank.  dist: 'normal' N(0,1), 'uniform' U[-1,1],
    'int' integers in [lo, hi] (inclusive), 'pow2' +-2^-1, +-1, +-2; cast to
    dtype."""
    g = rng_for(seed, rank)
    if dist == "normal":
        return cast(g.standard_normal(n), dtype)
    if dist == "uniform":
        return cast(g.uniform(-1.0, 1.0, n), dtype)
    if dist == "int":
        if dtype in INT_TYPES:
            # draw in the type's own width so that full 64-bit ranges work
            return g.integers(lo, hi, size=n, endpoint=True, dtype=NP_DTYPE[dtype])
        v = g.integers(lo, hi, size=n, endpoint=True)
        return cast(v.astype(np.float64), dtype)
    if dist == "pow2":   # +-2^e, e in [-1, 1]: products of a few are exact in every float type
        e = g.integers(-1, 1, size=n, endpoint=True).astype(np.float64)
        sgn = np.where(g.integers(0, 1, size=n, endpoint=True) == 1, 1.0, -1.0)
        return cast(sgn * np.exp2(e), dtype)
    raise ValueError(dist)


def workload(seed: int, k: int, n: int, dtype: str, dist: str = "normal", **kw):
    """Per-rank inputs of one collective: list of k arrays of n values."""
    return [rank_values(seed, r, n, dtype, dist, **kw) for r in range(k)]


def log_uniform_sizes(seed: int, m: int, lo_bytes: int, hi_bytes: int, align: int = 16):
    """m sizes log-uniform in [lo_bytes, hi_bytes], rounded down to `align`."""
    g = rng_for(seed, 10_000)
    e = g.uniform(math.log(lo_bytes), math.log(hi_bytes), m)
    s = (np.exp(e) // align).astype(np.int64) * align
    return np.maximum(s, align)
