"""Host-side checks that need no GPU: the library builds, loads and exports
every entry point declared in include/vcomm.h; arguments that are invalid
without touching the device are rejected; the ctypes binding declares the
same entry points as the header."""
import ctypes
import os
import re

import pytest

import paper_2507_04786_b300 as pkg
from paper_2507_04786_b300 import binding
from paper_2507_04786_b300 import build as vbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vcomm.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^(?:vResult_t|int)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    vbuild.build()
    return pkg.load_library()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 16
    raw = ctypes.CDLL(vbuild.OUT)
    for n in names:
        assert hasattr(raw, n), n
    assert sorted(binding.EXPORTS) == names


def test_version(lib):
    assert lib.vcommVersion() == 100


def test_host_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.vcommInit(None, 4, 1) == 1                      # vInvalidArgument
    assert lib.vcommInit(ctypes.byref(h), 0, 1) == 1
    assert lib.vcommInit(ctypes.byref(h), 65, 1) == 1
    assert lib.vcommInit(ctypes.byref(h), 4, 0) == 1
    assert lib.vcommInit(ctypes.byref(h), 4, 65) == 1
    assert lib.vcommSetPlan(None, None) == 1
    assert lib.vcommGetLastPlan(None, None) == 1
    assert lib.vcommDestroy(None) == 0
    arr = (ctypes.c_void_p * 4)()
    assert lib.vAllReduce(arr, arr, 10, 1, 0, 1, 1, None, None) == 1
    assert lib.vDebugEncode(1, None, 8, 1, None, None) == 1


def test_init_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.vcommInit(ctypes.byref(h), 4, 1)
    assert rc in (4, 2)            # vCudaError / vUnsupported, never a crash
    assert not h.value
