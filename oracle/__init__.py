"""CPU FP64 oracle for the block-Toeplitz F / F* matvecs.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the graft entry point's
smoke check and the benchmark's CPU-baseline leg, never by the GPU library.
It shares no code with the GPU path.  See :mod:`oracle.toeplitz`.
"""
from .toeplitz import *  # noqa: F401,F403
from .toeplitz import __all__  # noqa: F401
