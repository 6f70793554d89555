"""Thin Python binding of the C ABI in include/m2l.h (argument marshalling only).

Every function here forwards to the compiled library ``libm2l_gb300.so``; all arithmetic runs
in its CUDA kernels. Importing this module loads the library and raises ``ImportError`` if it
has not been built (``python -c "import __graft_entry__ as g; g.build()"``): there is no
CPU fallback.

Function names mirror the C ABI. ``Plan`` wraps a plan handle for use with torch tensors
(device memory and streams come from PyTorch).
"""

from __future__ import annotations

import ctypes
import os
import struct

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libm2l_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)

# enums (include/m2l.h)
M2L_LAPLACE3D = 0
M2L_OK, M2L_EINVAL, M2L_ENOMEM, M2L_ECUDA, M2L_ETIMEOUT, M2L_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
M2L_OPT_FORM, M2L_OPT_PRECISION, M2L_OPT_ACCUMULATE, M2L_OPT_OUTPUT, M2L_OPT_TARGET_TOL, M2L_OPT_FFT_GRID = 1, 2, 3, 4, 5, 6
M2L_OPT_TIMING = 7
M2L_OPT_TC_GROUP = 8
M2L_OPT_DIR_TOL = 9
M2L_OPT_CHECK_ORDER = 10
M2L_OPT_TC_CHUNK = 11
M2L_OPT_TC_DRAIN = 12
M2L_OPT_RANK_AUTO = 13
M2L_OPT_SVD = 14
M2L_OPT_HADAMARD_CHAINS = 15
M2L_Q_RANK_TOL = 17
M2L_Q_CONTRACT_FLOPS, M2L_Q_DIR_RANK_SUM, M2L_Q_NC, M2L_Q_RANK_CHECK = 13, 14, 15, 16
STAGES = ["compress", "contract", "expand", "fft_forward", "hadamard", "fft_inverse", "pinv"]
M2L_NUM_STAGES = 7
M2L_FORM_AUTO, M2L_FORM_BLAS, M2L_FORM_FFT = 0, 1, 2
M2L_PREC_AUTO, M2L_PREC_FP64, M2L_PREC_FP32, M2L_PREC_TF32X3, M2L_PREC_BF16X3 = -1, 0, 1, 2, 3
M2L_OUT_LOCALS, M2L_OUT_CHECK_POTENTIAL = 0, 1
(M2L_WAIT_GATHER, M2L_WAIT_TMA, M2L_WAIT_ACC_FREE, M2L_WAIT_OPERANDS, M2L_WAIT_ACC_READY,
 M2L_WAIT_SELFTEST) = range(1, 7)
(M2L_Q_N, M2L_Q_RANK, M2L_Q_BOXES, M2L_Q_PAIRS, M2L_Q_GRID, M2L_Q_FREQS, M2L_Q_PINV_RANK, M2L_Q_ROWS,
 M2L_Q_FORM, M2L_Q_PRECISION, M2L_Q_LAUNCHES, M2L_Q_DEVICE_STATUS) = range(1, 13)

FORMS = {"auto": M2L_FORM_AUTO, "blas": M2L_FORM_BLAS, "fft": M2L_FORM_FFT}
PRECISIONS = {"auto": M2L_PREC_AUTO, "fp64": M2L_PREC_FP64, "fp32": M2L_PREC_FP32,
              "tf32x3": M2L_PREC_TF32X3, "bf16x3": M2L_PREC_BF16X3}

_vp = ctypes.c_void_p
_lib.m2l_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
_lib.m2l_plan.restype = _vp
_lib.m2l_apply.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int]
_lib.m2l_apply.restype = ctypes.c_int
_lib.m2l_destroy.argtypes = [_vp]
_lib.m2l_destroy.restype = None
_lib.m2l_last_error.argtypes = []
_lib.m2l_last_error.restype = ctypes.c_char_p
_lib.m2l_set_option.argtypes = [_vp, ctypes.c_int, ctypes.c_longlong]
_lib.m2l_set_option.restype = ctypes.c_int
_lib.m2l_set_stream.argtypes = [_vp, _vp]
_lib.m2l_set_stream.restype = ctypes.c_int
_lib.m2l_set_boxes.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_longlong]
_lib.m2l_set_boxes.restype = ctypes.c_int
_lib.m2l_apply_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                 ctypes.POINTER(ctypes.c_int)]
_lib.m2l_apply_batch.restype = ctypes.c_int
_lib.m2l_query.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
_lib.m2l_query.restype = ctypes.c_int
_lib.m2l_stage_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
_lib.m2l_stage_times.restype = ctypes.c_int
_lib.m2l_apply_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int]
_lib.m2l_apply_noalloc.restype = ctypes.c_int
_lib.m2l_get_operator.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
_lib.m2l_get_operator.restype = ctypes.c_int
_lib.m2l_selftest_watchdog.argtypes = [_vp, ctypes.c_longlong]
_lib.m2l_selftest_watchdog.restype = ctypes.c_int
_dpp = ctypes.POINTER(ctypes.c_double)
_lib.m2l_fmm_plan.argtypes = [_dpp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dpp, ctypes.c_double]
_lib.m2l_fmm_plan.restype = _vp
_lib.m2l_fmm_set_m2l_option.argtypes = [_vp, ctypes.c_int, ctypes.c_longlong]
_lib.m2l_fmm_set_m2l_option.restype = ctypes.c_int
_lib.m2l_fmm_evaluate.argtypes = [_vp, _vp, _vp]
_lib.m2l_fmm_evaluate.restype = ctypes.c_int
_lib.m2l_fmm_m2l_plan.argtypes = [_vp]
_lib.m2l_fmm_m2l_plan.restype = _vp
_lib.m2l_fmm_destroy.argtypes = [_vp]
_lib.m2l_fmm_destroy.restype = None


class M2LError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"m2l error {code}: {msg}")
        self.code = code


def m2l_last_error() -> str:
    return (_lib.m2l_last_error() or b"").decode()


def _check(rc: int) -> int:
    if rc != M2L_OK:
        raise M2LError(rc, m2l_last_error())
    return rc


def m2l_plan(depth: int, p: int, kernel: int = M2L_LAPLACE3D, rank_tol: float = 0.0) -> int:
    h = _lib.m2l_plan(depth, p, kernel, rank_tol)
    if not h:
        raise M2LError(M2L_EINVAL, m2l_last_error())
    return h


def m2l_apply(plan, multipoles_ptr: int, locals_ptr: int, level: int, n_rhs: int) -> int:
    return _lib.m2l_apply(plan, multipoles_ptr, locals_ptr, level, n_rhs)


def m2l_apply_noalloc(plan, multipoles_ptr: int, locals_ptr: int, level: int, n_rhs: int) -> int:
    """FP64 BLAS form at one level with the library's static scratch: allocates nothing (include/m2l.h)."""
    return _lib.m2l_apply_noalloc(plan, multipoles_ptr, locals_ptr, level, n_rhs)


def m2l_destroy(plan) -> None:
    _lib.m2l_destroy(plan)


def m2l_set_option(plan, key: int, value) -> int:
    if key in (M2L_OPT_TARGET_TOL, M2L_OPT_DIR_TOL):
        value = struct.unpack("<q", struct.pack("<d", float(value)))[0]
    return _lib.m2l_set_option(plan, key, int(value))


def m2l_set_stream(plan, stream_ptr: int) -> int:
    return _lib.m2l_set_stream(plan, stream_ptr)


def m2l_set_boxes(plan, level: int, keys_ptr, n: int) -> int:
    return _lib.m2l_set_boxes(plan, level, keys_ptr, n)


def m2l_apply_batch(plans, multipoles_ptrs, locals_ptrs, n_rhs) -> int:
    k = len(plans)
    P = (_vp * k)(*plans)
    Q = (_vp * k)(*multipoles_ptrs)
    L = (_vp * k)(*locals_ptrs)
    R = (ctypes.c_int * k)(*n_rhs)
    return _lib.m2l_apply_batch(P, k, Q, L, R)


def m2l_query(plan, what: int, level: int = -1) -> int:
    out = ctypes.c_longlong(0)
    _check(_lib.m2l_query(plan, what, level, ctypes.byref(out)))
    return out.value


def m2l_device_status(plan) -> int:
    """The plan's device status word (0, or the M2L_WAIT_* code of a bounded wait that ran out),
    read and cleared without raising; m2l_query(M2L_Q_DEVICE_STATUS) raises M2LError(M2L_ETIMEOUT)
    for a nonzero word instead."""
    out = ctypes.c_longlong(0)
    rc = _lib.m2l_query(plan, M2L_Q_DEVICE_STATUS, -1, ctypes.byref(out))
    if rc not in (M2L_OK, M2L_ETIMEOUT):
        _check(rc)
    return out.value


def m2l_selftest_watchdog(plan, polls: int) -> None:
    _check(_lib.m2l_selftest_watchdog(plan, polls))


def m2l_stage_times(plan):
    """{stage name: (milliseconds, launches)} of the last timed application."""
    ms = (ctypes.c_double * M2L_NUM_STAGES)()
    ln = (ctypes.c_longlong * M2L_NUM_STAGES)()
    _check(_lib.m2l_stage_times(plan, ms, ln))
    return {STAGES[i]: (ms[i], ln[i]) for i in range(M2L_NUM_STAGES)}


def m2l_get_operator(plan, which: int):
    import numpy as np
    cnt = ctypes.c_longlong(0)
    _check(_lib.m2l_get_operator(plan, which, None, ctypes.byref(cnt)))
    buf = np.zeros(cnt.value, dtype=np.float64)
    _check(_lib.m2l_get_operator(plan, which, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt)))
    return buf


_lib.m2l_stated_bound.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
_lib.m2l_stated_bound.restype = ctypes.c_int


def m2l_stated_bound(form: int, precision: int, p: int) -> float:
    out = ctypes.c_double(0.0)
    _check(_lib.m2l_stated_bound(form, precision, p, ctypes.byref(out)))
    return out.value


class Plan:
    """A plan handle bound to torch tensors (device or host) and the current torch stream."""

    def __init__(self, depth: int, p: int, rank_tol: float = 0.0, form: str = "blas", precision: str = "fp64"):
        self.depth, self.p, self.rank_tol = depth, p, rank_tol
        self.handle = m2l_plan(depth, p, M2L_LAPLACE3D, rank_tol)
        self.set(form=form, precision=precision)

    def set(self, form=None, precision=None, accumulate=None, output=None, target_tol=None, fft_grid=None,
            timing=None, tc_group=None, dir_tol=None, check_order=None, tc_chunk=None, tc_drain=None,
            rank_auto=None, svd=None, had_chains=None):
        if form is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_FORM, FORMS[form]))
        if precision is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_PRECISION, PRECISIONS[precision]))
        if accumulate is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_ACCUMULATE, int(bool(accumulate))))
        if output is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_OUTPUT,
                                  {"locals": M2L_OUT_LOCALS, "check": M2L_OUT_CHECK_POTENTIAL}[output]))
        if target_tol is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_TARGET_TOL, target_tol))
        if fft_grid is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_FFT_GRID, fft_grid))
        if timing is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_TIMING, int(bool(timing))))
        if tc_group is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_TC_GROUP, int(tc_group)))
        if dir_tol is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_DIR_TOL, float(dir_tol)))
        if check_order is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_CHECK_ORDER, int(check_order)))
        if tc_chunk is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_TC_CHUNK, int(tc_chunk)))
        if tc_drain is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_TC_DRAIN, int(tc_drain)))
        if rank_auto is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_RANK_AUTO, int(bool(rank_auto))))
        if svd is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_SVD, {"exact": 0, "randomised": 1}[svd]))
        if had_chains is not None:
            _check(m2l_set_option(self.handle, M2L_OPT_HADAMARD_CHAINS, int(had_chains)))
        return self

    def stage_times(self):
        return m2l_stage_times(self.handle)

    def set_boxes(self, level: int, keys) -> None:
        """keys: sorted uint64 Morton keys (numpy), or None for the full level."""
        import numpy as np
        if keys is None:
            _check(m2l_set_boxes(self.handle, level, None, 8 ** level))
            return
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        _check(m2l_set_boxes(self.handle, level, k.ctypes.data, len(k)))

    def set_stream(self, stream=None) -> None:
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        _check(m2l_set_stream(self.handle, s.cuda_stream))

    def query(self, what: int, level: int = -1) -> int:
        return m2l_query(self.handle, what, level)

    def current_rank_tol(self) -> float:
        """The plan's current rank threshold (as given, or as M2L_OPT_RANK_AUTO chose it)."""
        return struct.unpack("<d", struct.pack("<q", self.query(M2L_Q_RANK_TOL)))[0]

    @property
    def n(self) -> int:
        return self.query(M2L_Q_N)

    @property
    def nc(self) -> int:
        return self.query(M2L_Q_NC)

    def rows(self, level: int = -1) -> int:
        return self.query(M2L_Q_ROWS, level)

    def pairs(self, level: int = -1) -> int:
        return self.query(M2L_Q_PAIRS, level)

    def apply(self, multipoles, locals_, level: int = -1, n_rhs: int = 1) -> None:
        """multipoles / locals_: contiguous torch tensors (or numpy arrays) in the C-ABI layout."""
        qp = multipoles.data_ptr() if hasattr(multipoles, "data_ptr") else multipoles.ctypes.data
        lp = locals_.data_ptr() if hasattr(locals_, "data_ptr") else locals_.ctypes.data
        _check(m2l_apply(self.handle, qp, lp, level, n_rhs))

    def close(self) -> None:
        if getattr(self, "handle", None):
            m2l_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FMM:
    """A whole FMM (P2M, M2M, M2L, L2L, L2P, P2P on the GPU, FP64) over points fixed at plan time."""

    def __init__(self, points, depth: int, p: int, rank_tol: float = 0.0, origin=None, width: float = 1.0):
        import numpy as np
        pts = np.ascontiguousarray(points, dtype=np.float64)
        if pts.ndim != 2 or pts.shape[1] != 3:
            raise ValueError("points must be (N, 3)")
        self.n_points = pts.shape[0]
        org = None if origin is None else np.ascontiguousarray(origin, dtype=np.float64)
        self.handle = _lib.m2l_fmm_plan(pts.ctypes.data_as(_dpp), self.n_points, depth, p, rank_tol,
                                        None if org is None else org.ctypes.data_as(_dpp), width)
        if not self.handle:
            raise M2LError(M2L_EINVAL, m2l_last_error())

    def set_m2l(self, form=None, dir_tol=None, tc_group=None):
        if form is not None:
            _check(_lib.m2l_fmm_set_m2l_option(self.handle, M2L_OPT_FORM, FORMS[form]))
        if dir_tol is not None:
            bits = struct.unpack("<q", struct.pack("<d", float(dir_tol)))[0]
            _check(_lib.m2l_fmm_set_m2l_option(self.handle, M2L_OPT_DIR_TOL, bits))
        return self

    def m2l_query(self, what: int, level: int = -1) -> int:
        return m2l_query(_lib.m2l_fmm_m2l_plan(self.handle), what, level)

    def evaluate(self, charges, out=None):
        """Potentials at the points (numpy arrays on the host, or torch tensors on either side)."""
        import numpy as np
        if hasattr(charges, "data_ptr"):
            if out is None:
                out = charges.new_empty(charges.shape)
            _check(_lib.m2l_fmm_evaluate(self.handle, charges.data_ptr(), out.data_ptr()))
            return out
        q = np.ascontiguousarray(charges, dtype=np.float64)
        res = np.empty_like(q) if out is None else out
        _check(_lib.m2l_fmm_evaluate(self.handle, q.ctypes.data, res.ctypes.data))
        return res

    def close(self):
        if self.handle:
            _lib.m2l_fmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

