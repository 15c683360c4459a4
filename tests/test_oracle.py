"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
step tables retyped from the text, closed forms, the plain elementwise
definition on inputs where every association order gives the same bits,
library conversions (numpy, torch), hand-derived fold-order fixtures
(tests/golden/fold_order.json), rigorous floating-point error bounds, and
encode/decode round trips.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2507_04786_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------- step tables
# Retyped from the paper's tables (Sec. V-E).


def paper_ring_allreduce(k, t):
    # Table "Steps in one loop iteration of NCCL Ring AllReduce"
    if t == 0:
        return "send"
    if 1 <= t <= k - 2:
        return "recvReduceSend"
    if t == k - 1:
        return "recvReduceCopySend"
    if k <= t <= 2 * k - 3:
        return "recvCopySend"
    if t == 2 * k - 2:
        return "recv"
    return None


@pytest.mark.parametrize("k", list(range(2, 65)))
def test_ring_allreduce_table(k):
    got = [oracle.ring_prim("allreduce", k, t) for t in range(2 * k + 1)]
    want = [paper_ring_allreduce(k, t) for t in range(2 * k + 1)]
    assert got == want
    # 2k-1 steps per loop (Sec. V-E), 2(k-1) of them send to the FIFO and
    # 2(k-1) receive from it
    steps = [p for p in got if p]
    assert len(steps) == 2 * k - 1
    assert sum(1 for p in steps if p.endswith("Send") or p == "send") == 2 * (k - 1)
    assert sum(1 for p in steps if p.startswith("recv")) == 2 * (k - 1)


@pytest.mark.parametrize("k", list(range(2, 65)))
def test_ring_rs_ag_tables(k):
    # Tables "Ring ReduceScatter" and "Ring AllGather": k-1 FIFO hops each
    rs = [oracle.ring_prim("reducescatter", k, t) for t in range(k + 1)]
    assert rs[0] == "send" and rs[k - 1] == "recvReduceCopy" and rs[k] is None
    assert all(p == "recvReduceSend" for p in rs[1:k - 1])
    for inplace, first in ((True, "send"), (False, "copySend")):
        ag = [oracle.ring_prim("allgather", k, t, inplace) for t in range(k + 1)]
        assert ag[0] == first and ag[k - 1] == "recv" and ag[k] is None
        assert all(p == "recvCopySend" for p in ag[1:k - 1])
    assert sum(1 for p in rs if p and p != "recvReduceCopy") == k - 1


@pytest.mark.parametrize("k", [2, 3, 4, 7, 8, 16])
def test_chain_tables(k):
    # Tables "Ring Broadcast" (root, middle, last) and "Ring Reduce"
    # (initiator, middle, root); chains follow the ring r -> r+1
    for root in range(k):
        b = [oracle.chain_prim("broadcast", k, root, (root + p) % k) for p in range(k)]
        assert b[0] == "copySend" and b[-1] == "recv"
        assert oracle.chain_prim("broadcast", k, root, root, True) == "send"
        assert all(p == "recvCopySend" for p in b[1:-1])
        r = [oracle.chain_prim("reduce", k, root, (root + 1 + p) % k) for p in range(k)]
        assert r[0] == "send" and r[-1] == "recvReduceCopy"
        assert all(p == "recvReduceSend" for p in r[1:-1])
        # chain length k-1 hops
        assert sum(1 for p in r if p != "recvReduceCopy") == k - 1


# ---------------------------------------------------------------- double binary tree

def tree_struct(k, t):
    par, kids = {}, {}
    for r in range(k):
        p, c0, c1 = oracle.tree_links(k, t, r)
        par[r] = p
        kids[r] = [c for c in (c0, c1) if c >= 0]
    return par, kids


@pytest.mark.parametrize("k", list(range(1, 65)))
def test_double_binary_tree_properties(k):
    """Sec. II-C: no node is a non-leaf in both trees, at most one node is a
    leaf in both; tree B mirrors tree A for even k, shifts it by one for odd."""
    internal, leaves = [], []
    for t in (0, 1):
        par, kids = tree_struct(k, t)
        roots = [r for r in range(k) if par[r] < 0]
        assert roots == [oracle.tree_root(k, t)]
        # parent/child links agree and every rank is reached exactly once
        for r in range(k):
            assert len(kids[r]) <= 2
            for c in kids[r]:
                assert par[c] == r
        seen, stack, depth = set(), [(roots[0], 0)], 0
        while stack:
            r, d = stack.pop()
            assert r not in seen
            seen.add(r)
            depth = max(depth, d)
            stack.extend((c, d + 1) for c in kids[r])
        assert seen == set(range(k))
        # binary tree depth: floor(log2 k) for this construction
        assert depth == (int(math.floor(math.log2(k))) if k > 1 else 0)
        internal.append({r for r in range(k) if kids[r]})
        leaves.append({r for r in range(k) if not kids[r]})
    if k > 2:
        assert not (internal[0] & internal[1])
    assert len(leaves[0] & leaves[1]) <= 1
    if k > 1 and k % 2 == 1:
        assert len(leaves[0] & leaves[1]) == 1
    # mirror / shift relation
    parA, _ = tree_struct(k, 0)
    parB, _ = tree_struct(k, 1)
    for r in range(k):
        if k % 2 == 0:
            m = k - 1 - r
            pa = parA[m]
            assert parB[r] == (-1 if pa < 0 else k - 1 - pa)
        else:
            m = (r + 1) % k
            pa = parA[m]
            assert parB[r] == (-1 if pa < 0 else (pa - 1) % k)


def test_tree_depth_examples():
    # k=8: root rank 7 with the single child rank 3; depth 3.  k=16: depth 4.
    p, c0, c1 = oracle.tree_links(8, 0, 7)
    assert p == -1 and c0 == 3 and c1 == -1
    assert oracle.tree_prims(8, 0, 7) == ("recvReduceCopySend", None)
    assert oracle.tree_prims(8, 0, 3) == ("recvReduceSend", "recvCopySend")
    assert oracle.tree_prims(8, 0, 0) == ("send", "recv")


# ---------------------------------------------------------------- partition

def test_buffer_table():
    """Table "NCCL channel buffer sizes": slot capacity and effective data."""
    KiB = 1024
    assert oracle.slot_data_bytes("simple") == 512 * KiB
    assert oracle.slot_data_bytes("ll") == 16 * KiB
    assert oracle.slot_data_bytes("ll128") * 2 == 1125 * KiB  # 562.5 KiB
    assert 8 * oracle.DEFAULT_SLOT_BYTES["simple"] == 4 * 1024 * KiB
    assert 8 * oracle.DEFAULT_SLOT_BYTES["ll"] == 256 * KiB
    assert 8 * oracle.DEFAULT_SLOT_BYTES["ll128"] == 4800 * KiB
    assert oracle.chunk_units("simple", 4) == 131072
    assert oracle.chunk_units("ll128", 4) == 144000
    assert oracle.chunk_units("ll", 2) == 8192


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, 4097, 65536 + 3])
@pytest.mark.parametrize("ub", [1, 2, 4])
@pytest.mark.parametrize("C", [1, 2, 3, 4, 7, 32])
def test_channel_partition(n, ub, C):
    """Sec. V-C: channels own disjoint contiguous ranges (workOffset,
    channelCount) that cover the input in order; reading R1 balances them to
    within one 16-byte pack and gives the element tail to the last channel."""
    epp = 16 // ub
    pos, sizes = 0, []
    for ch in range(C):
        s, l = oracle.channel_range(n, ub, C, ch)
        assert s == pos and s % epp == 0
        pos += l
        sizes.append(l - (n % epp if ch == C - 1 else 0))
    assert pos == n
    assert max(sizes) - min(sizes) <= epp


def test_iteration_example():
    """Sec. V-C worked example (Fig. "iteration-data-split", text only): 2
    channels, chunkCount 2, loopCount 4; with one-element packs each channel
    runs its range in loops of 4 elements split into chunks of 2."""
    n, C, k, chunk, ub = 16, 2, 2, 2, 16       # 16-byte units: one element per pack
    starts = [oracle.channel_range(n, ub, C, ch) for ch in range(C)]
    assert starts == [(0, 8), (8, 8)]
    for s, l in starts:
        loops = list(range(s, s + l, k * chunk))
        assert len(loops) == 2
        for off in loops:
            assert oracle.ring_loop_chunk(off, s + l, k, chunk, ub) == chunk


def test_last_loop_split():
    # the last loop divides the remainder evenly over k segments, pack-rounded
    assert oracle.ring_loop_chunk(0, 100, 4, 64, 4) == 28   # ceil(100/4)=25 -> 28
    assert oracle.ring_loop_chunk(0, 4 * 64, 4, 64, 4) == 64


# ---------------------------------------------------------------- dtype codecs

def test_fp16_encoder_matches_numpy():
    g = np.random.default_rng(1)
    x = np.concatenate([
        g.standard_normal(20000) * 10.0 ** g.integers(-9, 6, 20000),
        [0.0, -0.0, 65504.0, 65519.99, 65520.0, -65520.0, 1e6, 2.0 ** -24, 2.0 ** -25,
         3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11,
         np.inf, -np.inf]])
    got = oracle.encode("fp16", x).view(np.uint16)
    want = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want)
    back = oracle.decode("fp16", got.view(np.float16))
    assert np.array_equal(back[np.isfinite(back)], want.view(np.float16).astype(np.float64)[np.isfinite(back)])


def test_fp32_encoder_matches_numpy():
    g = np.random.default_rng(2)
    x = g.standard_normal(20000) * 10.0 ** g.integers(-45, 38, 20000)
    x = np.concatenate([x, [1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 2.0 ** -149, 2.0 ** -150,
                            3 * 2.0 ** -151, 3.4028235677973366e38, 3.5e38]])
    with np.errstate(over="ignore"):
        want = x.astype(np.float32).view(np.uint32)
    got = oracle.encode("fp32", x).view(np.uint32)
    assert np.array_equal(got, want)


def test_bf16_encoder_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(3)
    # fp32-representable inputs so torch's float -> bf16 path rounds once
    x = (g.standard_normal(20000) * 10.0 ** g.integers(-40, 38, 20000)).astype(np.float32)
    x = np.concatenate([x, np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 2.0 ** -133, 2.0 ** -134,
                                     3.3895314e38, 3.39e38, -0.0], np.float32)])
    got = oracle.encode("bf16", x.astype(np.float64))
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, want)


# ---------------------------------------------------------------- brute force

def plain_reduce(xs, dtype, op):
    """The order-free definition: elementwise sum (two's-complement wrap for
    int32) or max, exact for the inputs used below."""
    if dtype == "int32":
        a = np.stack([x.astype(np.int64) for x in xs])
        if op == "sum":
            s = a.sum(axis=0)
            return ((s + 2 ** 31) % 2 ** 32 - 2 ** 31).astype(np.int32)
        return a.max(axis=0).astype(np.int32)
    a = np.stack([x.astype(np.float64) for x in xs])
    r = a.sum(axis=0) if op == "sum" else a.max(axis=0)
    return r.astype(xs[0].dtype)


def exact_inputs(seed, k, n, dtype, op):
    if dtype == "int32":
        # wide range so that int32 sums wrap around
        return inputs.workload(seed, k, n, "int32", "int", lo=-2 ** 31, hi=2 ** 31 - 1)
    # integers small enough that every partial sum is exact in fp32
    return inputs.workload(seed, k, n, "fp32", "int", lo=-1000, hi=1000)


TINY = [(k, n, C, chunk) for k in (1, 2, 3, 4, 5) for n in (1, 7, 16, 37, 64)
        for C in (1, 2, 4) for chunk in (4, 8, 16)]


@pytest.mark.parametrize("k,n,C,chunk", TINY)
@pytest.mark.parametrize("dtype,op", [("int32", "sum"), ("int32", "max"), ("fp32", "sum"),
                                      ("fp32", "max")])
def test_brute_force_reductions(k, n, C, chunk, dtype, op):
    xs = exact_inputs(1000 * k + n, k, n, dtype, op)
    want = plain_reduce(xs, dtype, op)
    for algo in ("ring", "tree"):
        outs = oracle.all_reduce(xs, dtype, op, C, chunk, algo)
        for o in outs:
            assert np.array_equal(o, want), algo
    # ReduceScatter: block b of the plain reduction lands on rank b
    big = exact_inputs(7 + n, k, k * n, dtype, op)
    full = plain_reduce(big, dtype, op)
    rs = oracle.reduce_scatter(big, dtype, op, C, chunk)
    for b in range(k):
        assert np.array_equal(rs[b], full[b * n:(b + 1) * n])
    for root in range(k):
        assert np.array_equal(oracle.reduce(xs, dtype, op, root, C, chunk), want)


@pytest.mark.parametrize("k,n,C,chunk", TINY[::3])
def test_brute_force_copies(k, n, C, chunk):
    g = np.random.default_rng(k * 100 + n)
    xs = [g.integers(0, 256, n, dtype=np.uint8) for _ in range(k)]
    ag = oracle.all_gather(xs, C, chunk)
    want = np.concatenate(xs)
    for o in ag:
        assert np.array_equal(o, want)
    for root in range(k):
        for o in oracle.broadcast(xs, root, C, chunk):
            assert np.array_equal(o, xs[root])


# ---------------------------------------------------------------- fold order

def _golden():
    with open(os.path.join(GOLDEN, "fold_order.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_fold_order_golden(case):
    k = case["k"]
    n = case.get("count", case.get("recvcount", 0))
    if case["coll"] == "reducescatter":
        n *= k
    xs = [np.full(n, v, np.float16) for v in case["inputs"]]
    hexes = lambda a: [format(int(v), "04x") for v in a.view(np.uint16)]
    if case["coll"] == "allreduce":
        outs = oracle.all_reduce(xs, "fp16", "sum", case["nch"], case["chunk"], case["algo"],
                                 node=case.get("node", 1))
        for o in outs:
            assert hexes(o) == case["expected_hex"]
    elif case["coll"] == "reducescatter":
        outs = oracle.reduce_scatter(xs, "fp16", "sum", case["nch"], case["chunk"])
        for r, o in enumerate(outs):
            assert set(hexes(o)) == {case["expected_hex_per_rank"][r]}
    elif case["coll"] == "reduce":
        o = oracle.reduce(xs, "fp16", "sum", case["root"], case["nch"], case["chunk"])
        assert set(hexes(o)) == {case["expected_hex_root"]}


# ---------------------------------------------------------------- fp64 bounds

def unit_roundoff(dtype):
    return {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[dtype]


@pytest.mark.parametrize("dtype,dist", [("fp32", "normal"), ("bf16", "normal"),
                                        ("fp16", "uniform")])
@pytest.mark.parametrize("k", [2, 3, 8, 16])
@pytest.mark.parametrize("algo", ["ring", "tree"])
def test_fp64_error_bound(dtype, dist, k, algo):
    """Every element is a sum of k dtype values with k-1 roundings, so
    |y - sum| <= gamma_{k-1} * sum|x| with gamma_m = m u / (1 - m u); the
    normwise error stays within the 1e-6 (fp32) / 1e-2 (16-bit) target."""
    n = 5000 + 3
    xs = inputs.workload(11, k, n, dtype, dist)
    C, chunk = 3, 256
    outs = oracle.all_reduce(xs, dtype, "sum", C, chunk, algo)
    x64 = np.stack([oracle.decode(dtype, x) for x in xs])
    exact = x64.sum(axis=0)
    absum = np.abs(x64).sum(axis=0)
    u = unit_roundoff(dtype)
    m = k - 1
    gamma = m * u / (1 - m * u)
    y = oracle.decode(dtype, outs[0])
    # final rounding of an exactly representable... bound covers it: k-1 roundings total
    assert np.all(np.abs(y - exact) <= gamma * absum + 1e-300)
    tol = 1e-6 if dtype == "fp32" else 1e-2
    assert np.linalg.norm(y - exact) <= tol * np.linalg.norm(exact)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])      # all ranks bit-identical


def test_order_matters_for_fp():
    """Different plans give different (valid) fp bits: the oracle is not
    just a plain sum."""
    xs = inputs.workload(5, 8, 4096, "bf16", "normal")
    a = oracle.all_reduce(xs, "bf16", "sum", 1, 64, "ring")[0]
    b = oracle.all_reduce(xs, "bf16", "sum", 1, 64, "tree")[0]
    assert not np.array_equal(a, b)


# ---------------------------------------------------------------- encodings

@pytest.mark.parametrize("nbytes", [1, 3, 4, 5, 8, 119, 120, 121, 240, 1000, 16384])
def test_ll_round_trip(nbytes):
    """Sec. III-B: 4 data bytes + 4 flag bytes per 8-byte line."""
    g = np.random.default_rng(nbytes)
    d = g.integers(0, 256, nbytes, dtype=np.uint8)
    lines = oracle.ll_encode(d, 0xDEADBEEF)
    assert lines.size == (nbytes + 3) // 4
    assert np.all((lines >> np.uint64(32)) == 0xDEADBEEF)
    st, back = oracle.ll_decode(lines, nbytes, 0xDEADBEEF)
    assert st == 0 and np.array_equal(back, d)
    assert oracle.ll_decode(lines, nbytes, 0xDEADBEF0)[0] == 1      # stale flag
    bad = lines.copy()
    bad[-1] = bad[-1] & np.uint64(0xFFFFFFFF)
    assert oracle.ll_decode(bad, nbytes, 0xDEADBEEF)[0] == lines.size


@pytest.mark.parametrize("nbytes", [1, 8, 119, 120, 121, 480, 481, 576000])
def test_ll128_round_trip(nbytes):
    """Sec. III-C: 120 data bytes + an 8-byte flag per 128-byte line."""
    g = np.random.default_rng(nbytes)
    d = g.integers(0, 256, nbytes, dtype=np.uint8)
    flag = 0x0123456789ABCDEF
    lines = oracle.ll128_encode(d, flag)
    nl = (nbytes + 119) // 120
    assert lines.size == 16 * nl
    assert np.all(lines[15::16] == np.uint64(flag))
    raw = lines.view(np.uint8).reshape(nl, 128)
    assert np.array_equal(raw[:, :120].ravel()[:nbytes], d)
    st, back = oracle.ll128_decode(lines, nbytes, flag)
    assert st == 0 and np.array_equal(back, d)
    assert oracle.ll128_decode(lines, nbytes, flag + 1)[0] == 1


@pytest.mark.parametrize("algo", ["ring", "tree"])
@pytest.mark.parametrize("k,C,chunk,n", [(2, 1, 8, 100), (3, 2, 16, 1003), (8, 3, 64, 20011),
                                         (5, 4, 32, 4096)])
@pytest.mark.parametrize("dtype,op", [("fp32", "sum"), ("bf16", "sum"), ("fp16", "max")])
def test_point_queries_match_replay(algo, k, C, chunk, n, dtype, op):
    """The one-element queries used for full-size sampled checks agree with
    the full step-by-step replay on every element."""
    xs = inputs.workload(21, k, n, dtype, "normal")
    full = oracle.all_reduce(xs, dtype, op, C, chunk, algo)[0]
    pts = oracle.all_reduce_points(xs, np.arange(n), dtype, op, C, chunk, algo)
    assert np.array_equal(pts.view(np.uint8), full.view(np.uint8))


@pytest.mark.parametrize("k,C,chunk,n", [(2, 1, 8, 40), (3, 2, 16, 333), (8, 3, 64, 4001)])
@pytest.mark.parametrize("dtype,op", [("fp16", "sum"), ("bf16", "max"), ("int32", "sum")])
def test_rs_and_reduce_point_queries_match_replay(k, C, chunk, n, dtype, op):
    dist = "int" if dtype == "int32" else "normal"
    kw = {"lo": -2 ** 31, "hi": 2 ** 31 - 1} if dtype == "int32" else {}
    xs = inputs.workload(31, k, k * n, dtype, dist, **kw)
    rs = oracle.reduce_scatter(xs, dtype, op, C, chunk)
    for b in range(k):
        pts = oracle.reduce_scatter_points(xs, b, np.arange(n), dtype, op)
        assert np.array_equal(pts.view(np.uint8), rs[b].view(np.uint8))
    ys = [x[:n].copy() for x in xs]
    for root in (0, k - 1):
        full = oracle.reduce(ys, dtype, op, root, C, chunk)
        pts = oracle.reduce_points(ys, root, np.arange(n), dtype, op)
        assert np.array_equal(pts.view(np.uint8), full.view(np.uint8))


# ---------------------------------------------------------------- all-to-all and point-to-point

def test_all_to_all_hand_example():
    """Sec. II-A-4's all-to-all pattern, written out for 3 vranks x 2 elements
    per block: rank j receives block j of every rank, in rank order."""
    xs = [np.array([0, 1, 2, 3, 4, 5], dtype=np.int32) + 10 * r for r in range(3)]
    want = [[0, 1, 10, 11, 20, 21], [2, 3, 12, 13, 22, 23], [4, 5, 14, 15, 24, 25]]
    got = oracle.all_to_all(xs)
    for j in range(3):
        assert got[j].tolist() == want[j]


@pytest.mark.parametrize("k", [1, 2, 5, 9])
@pytest.mark.parametrize("dt", [np.float32, np.uint16, np.int32])
def test_all_to_all_is_an_involution(k, dt):
    rng = np.random.default_rng(k)
    n = 7
    xs = [rng.integers(0, 60000, k * n).astype(dt) for _ in range(k)]
    once = oracle.all_to_all(xs)
    twice = oracle.all_to_all(once)
    for r in range(k):
        assert np.array_equal(twice[r].view(np.uint8), xs[r].view(np.uint8))
        for j in range(k):   # block j of rank r's output is block r of rank j's input
            assert np.array_equal(once[r][j * n:(j + 1) * n], xs[j][r * n:(r + 1) * n])
    if k == 1:
        assert np.array_equal(once[0], xs[0])


def test_p2p_match_pairs_in_order():
    a0, a1, b0 = np.arange(3), np.arange(5) + 100, np.arange(2) + 7
    sends = [(0, 1, a0), (2, 1, b0), (0, 1, a1)]
    recvs = [(1, 0, 3), (1, 2, 2), (1, 0, 5)]
    got = oracle.p2p_match(sends, recvs)
    assert [g.tolist() for g in got] == [a0.tolist(), b0.tolist(), a1.tolist()]
    with pytest.raises(ValueError):
        oracle.p2p_match(sends, recvs[:2])                  # a send without its receive
    with pytest.raises(ValueError):
        oracle.p2p_match(sends, [(1, 0, 5), (1, 2, 2), (1, 0, 3)])   # counts cross
    with pytest.raises(ValueError):
        oracle.p2p_match(sends[:1], [(1, 0, 3), (0, 1, 3)])  # a receive without a send


# ---------------------------------------------------------------- more ops and dtypes (reading R18)

INT_BITS = {"int8": (8, True), "uint8": (8, False), "int32": (32, True), "uint32": (32, False),
            "int64": (64, True), "uint64": (64, False)}


def _wrap(v, dtype):
    bits, signed = INT_BITS[dtype]
    v %= 2 ** bits
    return v - 2 ** bits if signed and v >= 2 ** (bits - 1) else v


def _bf16_to_f64(bits):
    import torch
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).view(torch.bfloat16).double().numpy()


def plain_ext(xs, dtype, op, k):
    """Order-free definitions for the inputs below: Python integers for the
    integer types (wrap to the width; avg truncates toward zero), numpy
    min / max, and exact sums / products for the floats."""
    if dtype in INT_BITS:
        cols = zip(*[x.tolist() for x in xs])
        out = []
        for col in cols:
            if op in ("sum", "avg"):
                v = _wrap(sum(col), dtype)
                if op == "avg":
                    v = abs(v) // k * (1 if v >= 0 else -1)
            elif op == "prod":
                v = 1
                for c in col:
                    v = _wrap(v * c, dtype)
            else:
                v = max(col) if op == "max" else min(col)
            out.append(v)
        return np.array(out, dtype=xs[0].dtype)
    a = np.stack([_bf16_to_f64(x) if dtype == "bf16" else x.astype(np.float64) for x in xs])
    if op == "max":
        r = a.max(axis=0)
    elif op == "min":
        r = a.min(axis=0)
    elif op == "prod":
        r = a.prod(axis=0)
    else:
        r = a.sum(axis=0) / (k if op == "avg" else 1)
    return inputs.cast(r, dtype)


def ext_inputs(seed, k, n, dtype, op):
    if dtype in INT_BITS:
        bits, signed = INT_BITS[dtype]
        lo, hi = (-2 ** (bits - 1), 2 ** (bits - 1) - 1) if signed else (0, 2 ** bits - 1)
        return inputs.workload(seed, k, n, dtype, "int", lo=lo, hi=hi)
    if op == "prod":
        return inputs.workload(seed, k, n, dtype, "pow2")
    if op in ("max", "min"):
        return inputs.workload(seed, k, n, dtype, "normal")
    # integers whose every partial sum is exact in the type
    lim = {"fp64": 10 ** 6, "fp32": 1000, "fp16": 200, "bf16": 50}[dtype]
    return inputs.workload(seed, k, n, dtype, "int", lo=-lim, hi=lim)


EXT_TYPES = ["int8", "uint8", "int32", "uint32", "int64", "uint64", "fp16", "bf16", "fp32", "fp64"]


@pytest.mark.parametrize("k,n,C,chunk", [(1, 17, 1, 16), (2, 64, 3, 16), (3, 17, 1, 32),
                                         (5, 64, 3, 16), (4, 33, 2, 32)])
@pytest.mark.parametrize("dtype", EXT_TYPES)
@pytest.mark.parametrize("op", ["sum", "prod", "max", "min", "avg"])
def test_brute_force_ops_and_dtypes(k, n, C, chunk, dtype, op):
    xs = ext_inputs(977 * k + n, k, n, dtype, op)
    want = plain_ext(xs, dtype, op, k)
    for algo in ("ring", "tree"):
        for o in oracle.all_reduce(xs, dtype, op, C, chunk, algo):
            assert np.array_equal(o.view(np.uint8), want.view(np.uint8)), algo
    big = ext_inputs(5 + n, k, k * n, dtype, op)
    full = plain_ext(big, dtype, op, k)
    rs = oracle.reduce_scatter(big, dtype, op, C, chunk)
    for b in range(k):
        assert np.array_equal(rs[b].view(np.uint8), full[b * n:(b + 1) * n].view(np.uint8))
    for root in range(k):
        got = oracle.reduce(xs, dtype, op, root, C, chunk)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8))


def test_avg_divides_once_at_the_end():
    """avg is the sum divided by k once: 3 ranks of fp32 1.0 give 1.0 (an avg
    that divided on every hop would give (1/3 + 1)/3 + 1 ...), and the integer
    form truncates toward zero."""
    xs = [np.ones(5, dtype=np.float32) for _ in range(3)]
    for algo in ("ring", "tree"):
        for o in oracle.all_reduce(xs, "fp32", "avg", 1, 16, algo):
            assert o.tolist() == [1.0] * 5
    ys = [np.array([-7, 7, -8, 8], dtype=np.int32), np.array([0, 0, 0, 0], dtype=np.int32)]
    assert oracle.all_reduce(ys, "int32", "avg", 1, 16)[0].tolist() == [-3, 3, -4, 4]
    zs = [np.array([1.0, 2.0], dtype=np.float64) for _ in range(3)]
    assert oracle.reduce(zs, "fp64", "avg", 1, 1, 2).tolist() == [1.0, 2.0]


@pytest.mark.parametrize("dtype,op", [("fp64", "sum"), ("fp32", "prod"), ("bf16", "avg"),
                                      ("int8", "sum"), ("uint64", "min"), ("fp16", "avg")])
def test_point_queries_match_replay_new_ops(dtype, op):
    k, C, chunk, n = 5, 3, 32, 3001
    dist = "int" if dtype in INT_BITS else ("pow2" if op == "prod" else "normal")
    kw = {}
    if dtype in INT_BITS:
        bits, signed = INT_BITS[dtype]
        kw = {"lo": -2 ** (bits - 1) if signed else 0, "hi": 2 ** (bits - 1) - 1 if signed else 2 ** bits - 1}
    xs = inputs.workload(41, k, n, dtype, dist, **kw)
    for algo in ("ring", "tree"):
        full = oracle.all_reduce(xs, dtype, op, C, chunk, algo)[0]
        pts = oracle.all_reduce_points(xs, np.arange(n), dtype, op, C, chunk, algo)
        assert np.array_equal(pts.view(np.uint8), full.view(np.uint8)), algo
    for root in (0, k - 1):
        full = oracle.reduce(xs, dtype, op, root, C, chunk)
        pts = oracle.reduce_points(xs, root, np.arange(n), dtype, op)
        assert np.array_equal(pts.view(np.uint8), full.view(np.uint8))


# ---------------------------------------------------------------- hierarchical tree (reading R19)

HT = [(m, n) for m in (1, 2, 3, 4, 5) for n in range(1, 10)]


@pytest.mark.parametrize("m,nn", HT)
def test_hierarchical_tree_structure(m, nn):
    """Sec. V-E: branching only across nodes, a chain inside each node; every
    rank has at most two children; one root; the node graph is the double
    binary tree over the nodes; m = 1 is the flat tree."""
    k = m * nn
    for t in (0, 1):
        links = [oracle.htree_links(k, m, t, r) for r in range(k)]
        roots = [r for r in range(k) if links[r][0] < 0]
        assert roots == [oracle.htree_root(k, m, t)] and roots[0] % m == 0
        seen, stack = set(), [roots[0]]
        while stack:                                   # a tree: every rank reached once
            r = stack.pop()
            assert r not in seen
            seen.add(r)
            for c in links[r][1:]:
                if c >= 0:
                    assert links[c][0] == r
                    stack.append(c)
        assert seen == set(range(k))
        for r, (p, c0, c1) in enumerate(links):
            i = r % m
            if i > 0:
                assert p == r - 1                      # chain inside the node
            if i < m - 1:
                assert (c0, c1) == (r + 1, -1)
            else:
                for c in (c0, c1):                     # branches leave from a node's last rank
                    assert c < 0 or (c % m == 0 and c // m != r // m)
            if m == 1:
                assert (p, c0, c1) == oracle.tree_links(k, t, r)
        # node graph = the flat double binary tree over the nodes
        if nn > 1:
            for node in range(nn):
                p_node, a, b = oracle.tree_links(nn, t, node)
                first, last = node * m, node * m + m - 1
                assert links[first][0] == (p_node * m + m - 1 if p_node >= 0 else -1)
                assert [c // m for c in links[last][1:] if c >= 0] == [c for c in (a, b) if c >= 0]


@pytest.mark.parametrize("m,nn", [(2, 2), (2, 3), (3, 3), (4, 2), (5, 1)])
@pytest.mark.parametrize("dtype,op", [("int32", "sum"), ("int64", "max"), ("uint8", "prod"),
                                      ("fp32", "min"), ("int8", "avg")])
def test_hierarchical_tree_brute_force(m, nn, dtype, op):
    k, n = m * nn, 37
    xs = ext_inputs(11 * k + m, k, n, dtype, op)
    want = plain_ext(xs, dtype, op, k)
    for o in oracle.all_reduce(xs, dtype, op, 2, 16, "tree", node=m):
        assert np.array_equal(o.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("m,nn", [(2, 4), (4, 2), (3, 5)])
def test_hierarchical_tree_points_match_replay(m, nn):
    k, n = m * nn, 2003
    xs = inputs.workload(3, k, n, "bf16", "normal")
    full = oracle.all_reduce(xs, "bf16", "sum", 3, 64, "tree", node=m)[0]
    pts = oracle.all_reduce_points(xs, np.arange(n), "bf16", "sum", 3, 64, "tree", node=m)
    assert np.array_equal(pts.view(np.uint8), full.view(np.uint8))
