"""vcomm: virtual-rank ring / tree collectives on one B300 (sm_103a).

The compute path is the CUDA library ``libvcomm.so`` built from ``csrc/``
and reached through the C ABI in ``include/vcomm.h``; ``binding`` marshals
arguments to it with ctypes.  PyTorch is used only for device memory and
streams.  There is no CPU fallback: a missing library raises at first use.
"""
from .binding import (  # noqa: F401
    Comm, Server, VcommError, group, lib_path, load_library, version,
)
