"""Binding of the benchmark's measurement probes (libcagra_probes.so,
include/cagra_probes.h): the roofline denominators of the gathers, measured
on the GPU at hand.  Not part of the product library."""
from __future__ import annotations

import ctypes
import os
import threading

from .cagra import CagraError, _stream

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcagra_probes.so")
EXPORTS = ["cg_measure_row_gather", "cg_measure_smem_lookups"]
_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise CagraError(f"probe library not found at {p}; build it with "
                             "paper_1608_01362_gb300.build.build()")
        lib = ctypes.CDLL(p)
        lib.cg_measure_row_gather.restype = ctypes.c_int
        lib.cg_measure_row_gather.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                              ctypes.c_void_p]
        lib.cg_measure_smem_lookups.restype = ctypes.c_int
        lib.cg_measure_smem_lookups.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.cg_last_error_message.restype = ctypes.c_char_p
        lib.cg_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != 0:
        lib = load()
        raise CagraError(f"{what}: {lib.cg_status_string(status).decode()}: "
                         f"{lib.cg_last_error_message().decode(errors='replace')}")


def measure_row_gather(row_bytes: int, table_bytes: int, stream=None) -> float:
    """Bytes per second of random row reads (rows of row_bytes from a table of
    table_bytes; L2-resident or not) by a GPU-filling grid."""
    out = ctypes.c_double()
    _check(load().cg_measure_row_gather(row_bytes, int(table_bytes), ctypes.byref(out),
                                        _stream(stream)), "cg_measure_row_gather")
    return out.value


def measure_smem_lookups(stream=None) -> float:
    """Random 4-byte shared-memory lookups per second over the whole GPU."""
    out = ctypes.c_double()
    _check(load().cg_measure_smem_lookups(ctypes.byref(out), _stream(stream)),
           "cg_measure_smem_lookups")
    return out.value
