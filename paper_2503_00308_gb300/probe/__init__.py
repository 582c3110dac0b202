"""The benchmark's FP32 FMA-rate helper (libarprobe.so, built by _build.build).

A measurement utility for the render kernel's roofline: the FP32 FMA rate of
the current device.  It is a library of its own, not part of libar or of the
rendering path.
"""
from __future__ import annotations

import ctypes
import os

from .. import _build

_lib = None


def fp32_fma_rate(packed: bool, iters: int = 16384, stream=0) -> float:
    """TFLOP/s of 16 independent FMA chains per thread (packed: in pairs), timed on `stream`."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.PROBE_LIB):
            raise RuntimeError("libarprobe.so is not built; call __graft_entry__.build()")
        _lib = ctypes.CDLL(_build.PROBE_LIB)
        _lib.arprobe_fp32_fma_rate.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        _lib.arprobe_fp32_fma_rate.restype = ctypes.c_int
    v = ctypes.c_double(0.0)
    if _lib.arprobe_fp32_fma_rate(1 if packed else 0, int(iters), ctypes.byref(v), stream or None):
        raise RuntimeError("FMA rate probe failed (bad arguments or a CUDA error)")
    return v.value
