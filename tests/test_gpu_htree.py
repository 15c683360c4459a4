"""GPU parity of the hierarchical tree AllReduce (Sec. V-E: the double binary
tree branches only across nodes; inside a node the vranks form a chain),
bit-exact against the oracle's replay for every FIFO protocol, single and
grouped calls."""
import pytest

import oracle
from paper_2507_04786_b300 import Comm, VcommError, group, inputs

from gpu_util import SMALL_SLOTS, assert_same, chunk_for, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIST = {"fp32": ("normal", {}), "bf16": ("normal", {}), "int32": ("int", {"lo": -2 ** 20, "hi": 2 ** 20})}


def data(seed, k, n, dtype):
    dist, kw = DIST[dtype]
    return inputs.workload(seed, k, n, dtype, dist, **kw)


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128", "cluster"])
@pytest.mark.parametrize("k,m,C", [(8, 2, 1), (8, 4, 2), (6, 3, 1), (16, 4, 2), (4, 4, 1)])
@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "avg"), ("int32", "max")])
def test_hierarchical_tree_allreduce(proto, k, m, C, dtype, op):
    c = Comm(k, C, slot_bytes=SMALL_SLOTS, timeout_sec=10.0, tree_node=m)
    c.set_plan(nchannels=C, chunk_steps=1)
    for n in (1, 1001, 30011):
        xs = data(n + k + m, k, n, dtype)
        s = [to_dev(x) for x in xs]
        d = [torch.empty_like(t) for t in s]
        c.all_reduce(s, d, op=op, algo="tree", proto=proto)
        torch.cuda.synchronize()
        assert c.async_error() == "vSuccess"
        p = c.last_plan()
        assert p["algo"] == "tree"
        want = oracle.all_reduce(xs, dtype, op, C, chunk_for(proto, dtype, SMALL_SLOTS, 1), "tree", node=m)
        for r in (0, m - 1, k - 1):
            assert_same(to_np(d[r], dtype), want[r], f"{proto} k={k} m={m} n={n} rank {r}")
    c.destroy()


def test_hierarchical_tree_in_a_group():
    k, m = 8, 2
    c = Comm(k, 8, slot_bytes=SMALL_SLOTS, timeout_sec=10.0, tree_node=m)
    calls = []
    with group():
        for i, (dtype, n) in enumerate([("fp32", 5000), ("bf16", 777), ("int32", 20000)]):
            xs = data(40 + i, k, n, dtype)
            s = [to_dev(x) for x in xs]
            d = [torch.empty_like(t) for t in s]
            c.all_reduce(s, d, op="sum", algo="tree", proto="ll128")
            calls.append((dtype, xs, s, d))
    torch.cuda.synchronize()
    assert c.async_error() == "vSuccess"
    for (dtype, xs, _, d), p in zip(calls, c.group_plans()):
        want = oracle.all_reduce(xs, dtype, "sum", p["nchannels"],
                                 chunk_for(p["proto"], dtype, SMALL_SLOTS, p["chunkSteps"]), p["algo"],
                                 node=m if p["algo"] == "tree" else 1)
        for r in range(k):
            assert_same(to_np(d[r], dtype), want[r], f"{dtype} {p} rank {r}")
    c.destroy()


def test_node_size_must_divide_nranks():
    with pytest.raises(VcommError) as e:
        Comm(6, 1, tree_node=4)
    assert e.value.name == "vInvalidArgument"
