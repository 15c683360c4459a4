"""Build libvcomm.so in-tree with nvcc for sm_103a.

    python -m paper_2507_04786_b300.build [--force] [--verbose]

Compiles csrc/*.cu into objects under _build/ (in parallel; the reducing
kernel source is compiled once per (protocol, dtype) pair) and links one
shared library next to this file.  No fast-math and no FMA contraction: the
reductions must round exactly like IEEE adds.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build")
OUT = os.path.join(HERE, "libvcomm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
                 "-I", os.path.join(ROOT, "include"), "-I", CSRC]
# The batch kernel (vcomm_batch.cu) calls per-(protocol, dtype) worker
# functions compiled in vcomm_batch_inst.cu: those two units are relocatable
# device code, capped at the batch kernel's 128 registers; every other unit
# stays whole-program so its kernels keep their own inlining and launch bounds.
RDC = ["-rdc=true", "-maxrregcount=128"]
RDC_UNITS = ("vcomm_batch.cu", "vcomm_batch_inst.cu")
PER_PAIR = ("vcomm_reduce_inst.cu", "vcomm_batch_inst.cu")
PER_DTYPE = ("vcomm_cluster_inst.cu", "vcomm_direct_inst.cu")
NUM_DTYPES = 10   # vDataType_t


def units():
    """(source, object, extra flags) for every compilation unit."""
    out = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.splitext(os.path.basename(src))[0]
        extra = RDC if os.path.basename(src) in RDC_UNITS else []
        if os.path.basename(src) in PER_DTYPE:
            for d in range(NUM_DTYPES):
                out.append((src, os.path.join(OBJ, f"{base}_{d}.o"), extra + [f"-DVC_DTYPE={d}"]))
        elif os.path.basename(src) in PER_PAIR:
            for p in range(3):
                for d in range(NUM_DTYPES):
                    out.append((src, os.path.join(OBJ, f"{base}_{p}_{d}.o"),
                                extra + [f"-DVC_PROTO={p}", f"-DVC_DTYPE={d}"]))
        else:
            out.append((src, os.path.join(OBJ, base + ".o"), extra))
    return out


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) \
        + [os.path.join(ROOT, "include", "vcomm.h")]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + headers())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OBJ, exist_ok=True)
    todo = [(s, o, f) for (s, o, f) in units() if force or _stale(o, s)]
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(u):
        s, o, f = u
        cmd = [NVCC] + CFLAGS + extra + f + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return u, r

    failed = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
            for (s, o, f), r in ex.map(compile_one, todo):
                if verbose or r.returncode:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode:
                    failed.append(o)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    objs = [o for (_, o, _) in units()]
    if todo or not os.path.exists(OUT) or any(os.path.getmtime(o) > os.path.getmtime(OUT)
                                               for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-rdc=true", "-cudart", "static", "-o", OUT] + objs
        subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(OUT)
