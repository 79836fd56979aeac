"""Host-side checks of the C ABI: build, exported symbols, argument errors (no GPU work)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_10202_gb300 import build
    build.build()
    from paper_2508_10202_gb300 import _lib
    return _lib.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fftmv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fftmv_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["fftmv_create_operator", "fftmv_set_precision", "fftmv_matvec", "fftmv_rmatvec", "fftmv_free"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2508_10202_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_version_and_empty_error(lib):
    assert lib.fftmv_version() >= 100
    assert isinstance(lib.fftmv_last_error(), bytes)


def test_argument_errors(lib):
    h = ctypes.c_void_p()
    x = np.zeros((2, 2, 2))
    assert lib.fftmv_create_operator(None, 2, 2, 2, None, ctypes.byref(h)) == -1
    assert b"null" in lib.fftmv_last_error()
    assert lib.fftmv_create_operator(x.ctypes.data, 2, 2, 2, None, None) == -1
    for bad in [(0, 1, 1), (1, 0, 1), (1, 1, 0), (-3, 1, 1)]:
        assert lib.fftmv_create_operator(x.ctypes.data, *bad, None, ctypes.byref(h)) == -1
        assert b"sizes" in lib.fftmv_last_error()
    # Nt whose FFT length exceeds the shared-memory FFT
    assert lib.fftmv_create_operator(x.ctypes.data, 100000, 1, 1, None, ctypes.byref(h)) == -3
    assert b"exceeds" in lib.fftmv_last_error()


def test_null_and_dead_handles(lib):
    from paper_2508_10202_gb300 import _lib
    assert lib.fftmv_free(None) == 0
    fake = ctypes.c_void_p(0x1234)
    assert lib.fftmv_free(fake) == -5
    assert b"not live" in lib.fftmv_last_error()
    p = _lib.Precision(0, 0, 0, 0, 0, 0, 0)
    assert lib.fftmv_set_precision(fake, 0, ctypes.byref(p)) == -5
    assert lib.fftmv_matvec(fake, None, None, 1, 0, None) == -5
    assert lib.fftmv_matvec(None, None, None, 1, 0, None) == -1
    out = ctypes.c_size_t()
    assert lib.fftmv_workspace_bytes(fake, 0, 1, ctypes.byref(out)) == -5
    ms = (ctypes.c_double * 3)()
    assert lib.fftmv_phase_times(None, 0, ms, None) == -1
    assert lib.fftmv_check_bounded_wait(None, 10, 0, None) == -1
    assert lib.fftmv_check_bounded_wait(fake, 10, 0, None) == -5


def test_python_precision_strings():
    from paper_2508_10202_gb300 import make_precision
    p = make_precision("dssdd", "native")
    assert (p.pad, p.fft, p.gemv, p.ifft, p.unpad, p.gemv_mode, p.fft_mode) == (0, 1, 1, 0, 0, 0, 0)
    p = make_precision("ddddd", "f64x2f32")
    assert p.gemv_mode == 1 and p.fft_mode == 1
    p = make_precision("ddddd", "native", "f64x2f32")
    assert p.gemv_mode == 0 and p.fft_mode == 1
    with pytest.raises(ValueError):
        make_precision("dsdx")
    with pytest.raises(ValueError):
        make_precision("ddddd", "bogus")


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    x = np.zeros((2, 2, 2))
    h = ctypes.c_void_p()
    assert lib.fftmv_create_operator(x.ctypes.data, 2, 2, 2, None, ctypes.byref(h)) == -4
    assert h.value is None


def test_no_fallback_without_the_library(monkeypatch, tmp_path):
    # the package has no CPU path: with the shared library missing, creating
    # an operator raises ImportError instead of computing anything
    from paper_2508_10202_gb300 import Operator, _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libfftmv.so"))
    with pytest.raises(ImportError, match="no fallback"):
        _lib.lib()
    with pytest.raises(ImportError, match="no fallback"):
        Operator(np.zeros((2, 1, 1)))


def test_binding_rejects_bad_block_columns_before_any_call():
    # the Python binding checks dtype, rank and layout itself (no GPU needed)
    import torch
    from paper_2508_10202_gb300 import Operator
    with pytest.raises(ValueError, match="float64"):
        Operator(np.zeros((2, 3, 4), dtype=np.float32))      # FP32 block column
    with pytest.raises(ValueError, match="float64"):
        Operator(np.zeros((2, 3)))                            # not (Nt, Nd, Nm)
    with pytest.raises(TypeError, match="not supported"):
        Operator(np.zeros((2, 3, 4), dtype=np.int64))
    with pytest.raises(ValueError, match="contiguous"):
        Operator(np.zeros((4, 3, 2)).transpose(2, 1, 0))
    with pytest.raises(ValueError, match="contiguous"):
        Operator(torch.zeros((4, 3, 2), dtype=torch.float64).permute(2, 1, 0))
