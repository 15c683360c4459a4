"""bench.py on the CPU: the roofline's algorithmic bytes against the closed
forms of the ring AllReduce (2kS user bytes plus 4(k-1)S FIFO bytes, scaled
by each protocol's line overhead; 2kS without a FIFO), the bus-bandwidth
convention, and the reference arm's JSON line (it times the CPU oracle, so it
runs without a GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

S = 256 << 20


@pytest.mark.parametrize("proto,per_s", [("simple", 44.0), ("ll", 72.0),
                                         ("ll128", 16.0 + 28.0 * 128 / 120), ("direct", 16.0)])
def test_algorithmic_bytes_at_8_vranks(proto, per_s):
    assert bench.algorithmic_bytes(8, S, proto) == pytest.approx(per_s * S, rel=1e-12)


@pytest.mark.parametrize("k", [2, 3, 8, 16])
def test_algorithmic_bytes_closed_form(k):
    assert bench.algorithmic_bytes(k, S, "simple") == pytest.approx((2 * k + 4 * (k - 1)) * S)
    assert bench.algorithmic_bytes(k, S, "direct") == pytest.approx(2 * k * S)


def test_bus_bandwidth_convention():
    # AllReduce bus bandwidth = S / t x 2(k-1)/k
    assert bench.busbw(S, 8, 1e-3) == pytest.approx(S / 1e-3 * 2 * 7 / 8 / 1e9)
    assert bench.busbw(S, 2, 1e-3) == pytest.approx(S / 1e-3 / 1e9)


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "GB/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["config"]["workload"] == "ring-allreduce-8vr-256MiB"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("dtype,nch,n,proto", [("fp32", 37, 300_007, "simple"), ("bf16", 5, 123_457, "ll128"),
                                               ("fp32", 3, 70_001, "ll")])
def test_all_cores_oracle_equals_single_thread(dtype, nch, n, proto):
    """The CPU baseline's all-cores form (one oracle run per channel slice, on
    its own thread) gives the oracle's single-threaded bits."""
    import numpy as np

    import oracle
    from paper_2507_04786_b300 import inputs
    xs = inputs.workload(3, 8, n, dtype, "normal")
    es = oracle.ESIZE[dtype]
    chunk = oracle.chunk_units(proto, es, 1, {"simple": 8192, "ll": 2048, "ll128": 2560}[proto])
    one = bench.oracle_all_reduce(xs, dtype, "sum", nch, chunk, threads=1)
    many = bench.oracle_all_reduce(xs, dtype, "sum", nch, chunk, threads=4)
    for a, b in zip(one, many):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
