"""GB300-native FFT-based matvecs with block lower-triangular Toeplitz matrices.

The compute path is libfftmv.so (hand-written sm_103a CUDA behind a C ABI,
declared in include/fftmv.h); this package only marshals arguments.
"""
from ._lib import FftmvError, lib  # noqa: F401
from .operator import (Operator, create_operator, free, make_precision, matvec,  # noqa: F401
                       rmatvec, set_precision)

__all__ = ["Operator", "create_operator", "set_precision", "matvec", "rmatvec", "free",
           "make_precision", "FftmvError", "lib"]
