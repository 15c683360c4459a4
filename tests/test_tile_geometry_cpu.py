"""The tile engine's host-side geometry (vDebugTileGeometry; no GPU): how a
direct-protocol op is cut into tiles for group calls and serving mode 3.

Properties checked over a sweep of collectives, vrank counts, sizes, types
and access kinds:
* every byte of every block is in exactly one staged tile (perBlock tiles of
  tileBytes cover blockBytes), tiles are whole 4 KiB pieces, and one tile's
  HBM traffic stays within the 4 MiB cap;
* the staged bytes of a block are its full 16-byte units (ReduceScatter,
  AllReduce, Reduce, aligned copies) or, for an AllGather block that is not
  whole units, its aligned destination units but the last;
* a shifted window (blocks that are not whole units) never reads past the
  end of a send buffer, and an AllGather block's staged destination lies
  inside the block;
* the register path covers every unit with whole iterations, and its
  reductions go element by element;
* an op gets about two tiles per worker (whole pieces) unless the cap binds;
  a group launch's AllReduce tiles are at most 64 KiB.
"""
import numpy as np
import pytest

from paper_2507_04786_b300 import VcommError
from paper_2507_04786_b300 import build as vbuild
from paper_2507_04786_b300.binding import debug_tile_geometry

COPY = ("allgather", "broadcast")
BLOCKS = {"reducescatter": True, "allgather": True}
PIECE = 4096
CAP = 4 << 20
W = 147


@pytest.fixture(scope="module", autouse=True)
def lib():
    vbuild.build()


def factor(coll, k):
    return 2 * k if coll == "allreduce" else k + 1


def cases():
    rng = np.random.default_rng(11)
    out = []
    for coll in ("allreduce", "reducescatter", "allgather", "broadcast", "reduce"):
        for k in (1, 2, 3, 5, 8, 12, 16):
            for esz in ((1,) if coll in COPY else (2, 4)):
                for vec in (0, 1, 2):
                    if vec == 2 and coll not in BLOCKS:
                        continue
                    for _ in range(25):
                        count = int(rng.choice([1, 3, 15, 16, 17, 31, 33, 47, 48, 64, 1000, 4099, 65537,
                                                1 << 20, (1 << 20) + 3, 37 << 20, 301 << 20]))
                        if vec == 1 and coll in BLOCKS and (count * esz) % 16:
                            count = (count * esz + 15) // 16 * 16 // esz   # aligned blocks are whole units
                        if vec == 2 and (count * esz) % 16 == 0:
                            count += 1                                      # shifted blocks are not
                        out.append((coll, k, count, esz, vec))
    return out


CASES = cases()


def test_sweep_is_large():
    assert len(CASES) > 1000


def test_geometry_properties():
    for case in CASES:
        check(*case, shared=False)


def test_group_geometry_properties():
    """Group launches share tiles out statically: the same properties, with
    AllReduce tiles of at most 64 KiB."""
    for case in CASES:
        check(*case, shared=True)


def check(coll, k, count, esz, vec, shared):
    g = debug_tile_geometry(coll, k, count, esz, vec, W, 256, shared)
    copy = coll in COPY
    blocks = k if coll in BLOCKS else 1
    unit = 1 if copy else esz
    E = 16 // unit                       # elements (bytes) of a 16-byte unit
    assert g["ntiles"] >= 1
    # which bytes the staged path takes
    if vec == 1:
        want_block = (count // E) * 16
    elif vec == 2 and coll == "allgather":
        want_block = count // 16 * 16 - 16 if count >= 32 else 0
    elif vec == 2:
        want_block = (count // E) * 16
    else:
        want_block = 0
    staged = (vec == 1 and want_block >= 16) or (vec == 2 and want_block >= 32)
    assert g["staged"] == int(staged)
    if staged:
        B, T = g["blockBytes"], g["tileBytes"]
        assert B == want_block and B % 16 == 0
        assert T % PIECE == 0 and T >= PIECE
        assert g["perBlock"] == -(-B // T)                       # the tiles cover the block exactly
        assert (g["perBlock"] - 1) * T < B <= g["perBlock"] * T
        assert g["ntiles"] == blocks * g["perBlock"]
        assert T * factor(coll, k) <= max(CAP, PIECE * factor(coll, k))
        assert g["vec"] == vec
        C = count * unit                                         # bytes of a block
        if vec == 2 and coll == "allgather":
            for b in range(k):
                lead = (16 - (b * C) % 16) % 16                  # to the block's first aligned unit
                assert lead + B <= C                             # staged destination inside the block
                assert B + 16 <= C                               # the source window ends in the buffer
        if vec == 2 and coll == "reducescatter":
            for b in range(k):
                d = (b * C) % 16
                end = b * C - d + B + (16 if b < k - 1 else 0)   # the last block skips its last unit
                assert end <= k * C                              # the window ends in the send buffer
        # about two tiles per worker: the smallest whole-piece tile that gives
        # every worker at most two (unless the traffic cap binds first)
        share = -(-(blocks * B) // (2 * W))
        small = shared and coll == "allreduce"
        if small:
            assert T <= max(PIECE, 64 << 10)
        if (share + PIECE) * factor(coll, k) <= CAP and not (small and share > (64 << 10)):
            assert T >= share and (T == PIECE or T - PIECE < share)
    else:
        assert g["vec"] == (vec if copy else 0)                  # reductions: element by element
        if g["vec"] == 0:
            assert g["units"] == count * blocks
        assert g["tileUnits"] % 256 == 0
        assert g["ntiles"] == max(1, -(-g["units"] // g["tileUnits"]))


def test_refusals():
    with pytest.raises(VcommError):
        debug_tile_geometry("allreduce", 0, 10, 4, 1)
    with pytest.raises(VcommError):
        debug_tile_geometry("allreduce", 17, 10, 4, 1)
    with pytest.raises(VcommError):
        debug_tile_geometry("allreduce", 4, 10, 3, 1)
    with pytest.raises(VcommError):
        debug_tile_geometry("allreduce", 4, 10, 4, 3)
