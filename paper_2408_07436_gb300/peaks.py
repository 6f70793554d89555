"""Binding of the FMA-throughput probe in include/m2l_peaks.h (argument marshalling only).

The probe runs in ``libm2l_peaks.so``; importing this module raises ``ImportError`` when the
library has not been built.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libm2l_peaks.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA libraries first (__graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)
_dp = ctypes.POINTER(ctypes.c_double)
_lib.m2l_fma_peak.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, _dp, _dp, _dp]
_lib.m2l_fma_peak.restype = ctypes.c_int


def m2l_fma_peak(fp64: bool, iters: int, reps: int = 5):
    """(best, median) FMA throughput of the current device in TFLOP/s, and the best launch's ms."""
    best, med, ms = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    rc = _lib.m2l_fma_peak(int(bool(fp64)), int(iters), int(reps), ctypes.byref(best), ctypes.byref(med),
                           ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"m2l_fma_peak failed ({rc})")
    return best.value, med.value, ms.value
