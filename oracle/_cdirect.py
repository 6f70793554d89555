"""ctypes loader for oracle/direct.c (test infrastructure; see the package docstring).

``build()`` compiles the helper with gcc into ``oracle/_build``; ``lib()`` loads it, building
it first if it is missing.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_direct.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        ll = ctypes.POINTER(ctypes.c_longlong)
        _lib.oracle_check_potential.argtypes = [ctypes.c_int, ctypes.c_int, d, d, ctypes.c_longlong, d, ll, d, ll, d,
                                                ctypes.c_int, d]
        _lib.oracle_check_potential.restype = None
        _lib.oracle_direct_potential.argtypes = [ctypes.c_longlong, d, ctypes.c_longlong, d, d, d]
        _lib.oracle_direct_potential.restype = None
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


def check_potential(x_off, y_off, t_centre, offsets, s_centre, s_row, q, R):
    """phi[t, r, i] = sum over the sources e of target t of sum_j K(t_centre + x_off_i,
    s_centre_e + y_off_j) q[s_row_e, r, j]; x_off and y_off may have different lengths."""
    n = x_off.shape[0]
    ny = y_off.shape[0]
    x_off = np.ascontiguousarray(x_off, dtype=np.float64)
    y_off = np.ascontiguousarray(y_off, dtype=np.float64)
    t_centre = np.ascontiguousarray(t_centre, dtype=np.float64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    s_centre = np.ascontiguousarray(s_centre, dtype=np.float64).reshape(-1, 3)
    s_row = np.ascontiguousarray(s_row, dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    T = t_centre.shape[0]
    phi = np.zeros((T, R, n), dtype=np.float64)
    if T:
        lib().oracle_check_potential(n, ny, _dp(x_off), _dp(y_off), T, _dp(t_centre), _lp(offsets),
                                     _dp(s_centre), _lp(s_row), _dp(q), R, _dp(phi))
    return phi


def direct_potential(x, y, q):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(x.shape[0])
    lib().oracle_direct_potential(x.shape[0], _dp(x), y.shape[0], _dp(y), _dp(q), _dp(out))
    return out
