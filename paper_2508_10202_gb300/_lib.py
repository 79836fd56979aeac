"""ctypes declarations of the C ABI in include/fftmv.h.

The shared library is loaded from this package directory only; there is no
fallback implementation.  If it has not been built, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftmv.so")

FFTMV_OK = 0
STATUS = {0: "FFTMV_OK", -1: "FFTMV_EINVAL", -2: "FFTMV_ENOMEM", -3: "FFTMV_EUNSUPPORTED",
          -4: "FFTMV_ECUDA", -5: "FFTMV_ESTATE"}
FFTMV_F64, FFTMV_F32 = 0, 1
FFTMV_GEMV_NATIVE, FFTMV_GEMV_F64X2F32, FFTMV_GEMV_BF16X2, FFTMV_GEMV_F16X2 = 0, 1, 2, 3
FFTMV_FORWARD, FFTMV_ADJOINT = 0, 1
FFTMV_IO_F64, FFTMV_IO_F32 = 0, 1
FFTMV_STATUS_WAIT_TIMEOUT = 1


class FftmvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Precision(ctypes.Structure):
    _fields_ = [("pad", ctypes.c_int32), ("fft", ctypes.c_int32), ("gemv", ctypes.c_int32),
                ("ifft", ctypes.c_int32), ("unpad", ctypes.c_int32), ("gemv_mode", ctypes.c_int32),
                ("fft_mode", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("Nt", ctypes.c_int64), ("Nd", ctypes.c_int64), ("Nm", ctypes.c_int64),
                ("L", ctypes.c_int64), ("Nf", ctypes.c_int64), ("ldn", ctypes.c_int64),
                ("device", ctypes.c_int32), ("fhat_bytes", ctypes.c_size_t)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int

# name -> (restype, argtypes), the order of include/fftmv.h
SIGNATURES = {
    "fftmv_create_operator": (_INT, [_P, _I64, _I64, _I64, _P, ctypes.POINTER(_P)]),
    "fftmv_set_precision": (_INT, [_P, _INT, ctypes.POINTER(Precision)]),
    "fftmv_get_precision": (_INT, [_P, _INT, ctypes.POINTER(Precision)]),
    "fftmv_matvec": (_INT, [_P, _P, _P, _I64, _INT, _P]),
    "fftmv_rmatvec": (_INT, [_P, _P, _P, _I64, _INT, _P]),
    "fftmv_workspace_bytes": (_INT, [_P, _INT, _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "fftmv_set_scratch_limit": (_INT, [_P, ctypes.c_size_t]),
    "fftmv_set_fusion": (_INT, [_P, ctypes.c_int]),
    "fftmv_get_fhat": (_INT, [_P, _P, ctypes.c_size_t, _P]),
    "fftmv_create_from_fhat": (_INT, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, ctypes.POINTER(_P)]),
    "fftmv_apply_ws": (_INT, [_P, _INT, _P, _P, _I64, _INT, _P, ctypes.c_size_t, _P]),
    "fftmv_get_info": (_INT, [_P, ctypes.POINTER(Info)]),
    "fftmv_device_status": (_INT, [_P, ctypes.POINTER(ctypes.c_uint32), _INT]),
    "fftmv_check_bounded_wait": (_INT, [_P, ctypes.c_uint32, _INT, _P]),
    "fftmv_set_timing": (_INT, [_P, _INT]),
    "fftmv_phase_times": (_INT, [_P, _INT, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
    "fftmv_reset_timing": (_INT, [_P]),
    "fftmv_apply_noalloc": (_INT, [_P, _INT, _P, _P, _I64, _INT, _P]),
    "fftmv_free": (_INT, [_P]),
    "fftmv_last_error": (ctypes.c_char_p, []),
    "fftmv_version": (_INT, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libfftmv.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(or python -m paper_2508_10202_gb300.build); there is no fallback path")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(rc: int) -> None:
    if rc != FFTMV_OK:
        raise FftmvError(rc, lib().fftmv_last_error().decode(errors="replace"))
