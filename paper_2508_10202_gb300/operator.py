"""Python face of the C ABI: the same entry points, argument marshalling only.

Every step of a matvec runs in libfftmv.so's CUDA kernels.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays (host).  Host arrays go through
the library's host-I/O path (staged copies inside the call).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L

_PHASE_LETTERS = {"d": L.FFTMV_F64, "s": L.FFTMV_F32}
_MODES = {"native": L.FFTMV_GEMV_NATIVE, "f64x2f32": L.FFTMV_GEMV_F64X2F32, "bf16x2": L.FFTMV_GEMV_BF16X2,
          "f16x2": L.FFTMV_GEMV_F16X2}
_WHICH = {"F": L.FFTMV_FORWARD, "forward": L.FFTMV_FORWARD, L.FFTMV_FORWARD: L.FFTMV_FORWARD,
          "F*": L.FFTMV_ADJOINT, "adjoint": L.FFTMV_ADJOINT, L.FFTMV_ADJOINT: L.FFTMV_ADJOINT}


def make_precision(prec: str = "ddddd", mode: str = "native", fft_mode: str | None = None) -> L.Precision:
    """Precision struct from a 5-letter phase string over d/s (Section 3.2).

    ``mode`` is how an FP64 block matvec computes ("native" FP64 FMA or
    "f64x2f32" double-float); ``fft_mode`` the same for FP64 FFT/IFFT phases
    (defaults to ``mode``).
    """
    if len(prec) != 5 or any(c not in "ds" for c in prec):
        raise ValueError(f"precision must be 5 letters over d/s, got {prec!r}")
    if fft_mode is None:
        fft_mode = "f64x2f32" if mode == "f64x2f32" else "native"
    if mode not in _MODES or fft_mode not in _MODES:
        raise ValueError(f"modes must be among {sorted(_MODES)}")
    v = [_PHASE_LETTERS[c] for c in prec]
    return L.Precision(*v, _MODES[mode], _MODES[fft_mode])


def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _array_info(x):
    """(data pointer, io code, shape, is_cuda, device index)."""
    if _is_torch(x):
        torch = _torch()
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if x.dtype == torch.float64:
            io = L.FFTMV_IO_F64
        elif x.dtype == torch.float32:
            io = L.FFTMV_IO_F32
        else:
            raise TypeError(f"dtype {x.dtype} not supported (float64 or float32)")
        return x.data_ptr(), io, tuple(x.shape), x.is_cuda, (x.device.index if x.is_cuda else None)
    x = np.asarray(x)
    if not x.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    if x.dtype == np.float64:
        io = L.FFTMV_IO_F64
    elif x.dtype == np.float32:
        io = L.FFTMV_IO_F32
    else:
        raise TypeError(f"dtype {x.dtype} not supported (float64 or float32)")
    return x.ctypes.data, io, x.shape, False, None


def _stream_handle(stream, device) -> int:
    if stream is None:
        if device is None:
            return 0
        return _torch().cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


FHAT_HEADER_BYTES = 4096
_FHAT_FORMAT = "fftmv-fhat"


def fhat_header(Nt: int, Nd: int, Nm: int, L_: int, ldn: int) -> bytes:
    """The header block of a saved F-hat: JSON, space padded to FHAT_HEADER_BYTES."""
    import json
    h = json.dumps({"format": _FHAT_FORMAT, "version": 1, "Nt": int(Nt), "Nd": int(Nd), "Nm": int(Nm),
                    "L": int(L_), "Nf": int(L_) // 2 + 1, "ldn": int(ldn), "dtype": "complex128",
                    "layout": "[Nf][Nd][ldn], padding columns zero"}).encode()
    if len(h) >= FHAT_HEADER_BYTES:
        raise ValueError("header too long")
    return h + b" " * (FHAT_HEADER_BYTES - len(h))


def parse_fhat_header(block: bytes) -> dict:
    """Fields of a header block written by fhat_header (ValueError if it is not one)."""
    import json
    if len(block) != FHAT_HEADER_BYTES:
        raise ValueError("short header")
    try:
        h = json.loads(block.decode().rstrip(" "))
    except (UnicodeDecodeError, json.JSONDecodeError) as e:
        raise ValueError(f"not an F-hat file: {e}") from None
    if not isinstance(h, dict) or h.get("format") != _FHAT_FORMAT or h.get("version") != 1:
        raise ValueError("not an F-hat file (format/version)")
    for k in ("Nt", "Nd", "Nm", "L", "Nf", "ldn"):
        if not isinstance(h.get(k), int) or h[k] < 1:
            raise ValueError(f"bad header field {k}")
    if h["Nf"] != h["L"] // 2 + 1 or h["ldn"] < h["Nm"] or h["ldn"] % 8 or h["L"] < 2 * h["Nt"] - 1:
        raise ValueError("inconsistent header sizes")
    return h


def create_operator(F_col, stream=None) -> "Operator":
    """Operator from its first block column F_col[k, r, n] (FP64; host or device)."""
    return Operator(F_col, stream=stream)


class Operator:
    """A block lower-triangular Toeplitz operator resident on one GPU."""

    def __init__(self, F_col, stream=None):
        ptr, io, shape, is_cuda, dev = _array_info(F_col)
        if io != L.FFTMV_IO_F64 or len(shape) != 3:
            raise ValueError("F_col must be a float64 array of shape (Nt, Nd, Nm)")
        lib = L.lib()
        if is_cuda:
            _torch().cuda.set_device(dev)
        h = ctypes.c_void_p()
        L.check(lib.fftmv_create_operator(ptr, shape[0], shape[1], shape[2],
                                          _stream_handle(stream, dev), ctypes.byref(h)))
        self._attach(h)

    def _attach(self, h) -> None:
        self._h = h
        info = L.Info()
        L.check(L.lib().fftmv_get_info(self._h, ctypes.byref(info)))
        self.Nt, self.Nd, self.Nm = info.Nt, info.Nd, info.Nm
        self.L, self.Nf, self.ldn, self.device = info.L, info.Nf, info.ldn, info.device

    # -- checkpoint -----------------------------------------------------------
    def save(self, path, stream=None) -> None:
        """Write the master F-hat (fftmv_get_fhat) to ``path``: a header block
        (FHAT_HEADER_BYTES, JSON) and the [Nf][Nd][ldn] complex128 array."""
        nbytes = self.Nf * self.Nd * self.ldn * 16
        buf = np.empty(nbytes, dtype=np.uint8)
        L.check(L.lib().fftmv_get_fhat(self.handle, buf.ctypes.data, nbytes, _stream_handle(stream, None)))
        with open(path, "wb") as f:
            f.write(fhat_header(self.Nt, self.Nd, self.Nm, self.L, self.ldn))
            buf.tofile(f)

    @classmethod
    def load(cls, path, stream=None) -> "Operator":
        """Operator from a file written by ``save`` (fftmv_create_from_fhat: no
        setup FFT), on the current CUDA device."""
        with open(path, "rb") as f:
            hdr = parse_fhat_header(f.read(FHAT_HEADER_BYTES))
            n = hdr["Nf"] * hdr["Nd"] * hdr["ldn"] * 16
            data = np.fromfile(f, dtype=np.uint8, count=n)
        if data.size != n:
            raise ValueError(f"{path}: F-hat truncated ({data.size} of {n} bytes)")
        h = ctypes.c_void_p()
        L.check(L.lib().fftmv_create_from_fhat(data.ctypes.data, hdr["Nt"], hdr["Nd"], hdr["Nm"],
                                               _stream_handle(stream, None), ctypes.byref(h)))
        op = cls.__new__(cls)
        op._attach(h)
        if (op.L, op.ldn) != (hdr["L"], hdr["ldn"]):
            op.free()
            raise ValueError(f"{path}: saved with L={hdr['L']}, ldn={hdr['ldn']}; this library version uses "
                             f"L={op.L}, ldn={op.ldn} for Nt={hdr['Nt']}, Nm={hdr['Nm']}")
        return op

    # -- lifetime -----------------------------------------------------------
    def free(self) -> None:
        h, self._h = getattr(self, "_h", None), None
        if h:
            L.check(L.lib().fftmv_free(h))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise L.FftmvError(-5, "operator already freed")
        return self._h

    def info(self) -> L.Info:
        info = L.Info()
        L.check(L.lib().fftmv_get_info(self.handle, ctypes.byref(info)))
        return info

    # -- precision ------------------------------------------------------------
    def set_precision(self, which, prec: str = "ddddd", mode: str = "native", fft_mode: str | None = None) -> None:
        p = make_precision(prec, mode, fft_mode)
        L.check(L.lib().fftmv_set_precision(self.handle, _WHICH[which], ctypes.byref(p)))

    def get_precision(self, which) -> tuple[str, str, str]:
        p = L.Precision()
        L.check(L.lib().fftmv_get_precision(self.handle, _WHICH[which], ctypes.byref(p)))
        s = "".join("d" if v == L.FFTMV_F64 else "s" for v in (p.pad, p.fft, p.gemv, p.ifft, p.unpad))
        inv = {v: k for k, v in _MODES.items()}
        return s, inv[p.gemv_mode], inv[p.fft_mode]

    def workspace_bytes(self, which, K: int = 1) -> int:
        out = ctypes.c_size_t()
        L.check(L.lib().fftmv_workspace_bytes(self.handle, _WHICH[which], K, ctypes.byref(out)))
        return out.value

    def set_fusion(self, enable: bool = True) -> None:
        """Small all-FP64 and all-FP32 calls as one fused launch (fftmv_set_fusion; on by default)."""
        L.check(L.lib().fftmv_set_fusion(self.handle, int(bool(enable))))

    def set_scratch_limit(self, nbytes: int = 0) -> None:
        """Bound the pool scratch of one launch sequence; larger K runs in chunks (0: 8 GiB)."""
        L.check(L.lib().fftmv_set_scratch_limit(self.handle, int(nbytes)))

    # -- matvecs ------------------------------------------------------------
    def _apply(self, which: int, x, out, stream):
        n_in, n_out = (self.Nm, self.Nd) if which == L.FFTMV_FORWARD else (self.Nd, self.Nm)
        ptr, io, shape, is_cuda, dev = _array_info(x)
        if len(shape) == 2:
            K, out_shape = 1, (self.Nt, n_out)
        elif len(shape) == 3:
            K, out_shape = shape[0], (shape[0], self.Nt, n_out)
        else:
            raise ValueError("input must be (Nt, N) or (K, Nt, N)")
        if tuple(shape[-2:]) != (self.Nt, n_in):
            raise ValueError(f"input shape {shape} does not match (Nt={self.Nt}, N={n_in})")
        if out is None:
            if _is_torch(x):
                out = _torch().empty(out_shape, dtype=x.dtype, device=x.device)
            else:
                out = np.empty(out_shape, dtype=np.asarray(x).dtype)
        optr, oio, oshape, o_cuda, odev = _array_info(out)
        if tuple(oshape) != tuple(out_shape) or oio != io:
            raise ValueError(f"out must have shape {out_shape} and the input's dtype")
        dev = dev if dev is not None else odev
        fn = L.lib().fftmv_matvec if which == L.FFTMV_FORWARD else L.lib().fftmv_rmatvec
        L.check(fn(self.handle, ptr, optr, K, io, _stream_handle(stream, dev)))
        return out

    def apply_ws(self, which, x, out, workspace, stream=None):
        """F x or F* x into ``out`` with caller-owned scratch (a device uint8 tensor of at
        least workspace_bytes(which, K) bytes, 256-byte aligned); device tensors only."""
        w = _WHICH[which]
        ptr, io, shape, is_cuda, dev = _array_info(x)
        optr, oio, _, _, _ = _array_info(out)
        K = 1 if len(shape) == 2 else shape[0]
        L.check(L.lib().fftmv_apply_ws(self.handle, w, ptr, optr, K, io, workspace.data_ptr(),
                                       workspace.numel() * workspace.element_size(), _stream_handle(stream, dev)))
        return out

    def matvec(self, m, out=None, stream=None):
        """d = F m (Section 2.4): m is (Nt, Nm) or (K, Nt, Nm); returns (.., Nt, Nd).

        Device tensors, and host tensors that are all pinned, run stream ordered
        (synchronise the stream before reading ``out``); with a pageable host
        buffer the call returns with the result in place."""
        return self._apply(L.FFTMV_FORWARD, m, out, stream)

    def rmatvec(self, d, out=None, stream=None):
        """m = F* d (Section 2.4): d is (Nt, Nd) or (K, Nt, Nd); returns (.., Nt, Nm)."""
        return self._apply(L.FFTMV_ADJOINT, d, out, stream)

    def device_status(self, clear: bool = False) -> int:
        """Bits raised by device-side bounded waits (0 when every wait completed)."""
        v = ctypes.c_uint32()
        L.check(L.lib().fftmv_device_status(self.handle, ctypes.byref(v), int(bool(clear))))
        return v.value

    def check_bounded_wait(self, polls: int = 1000, complete: bool = False, stream=None) -> None:
        """Run the bounded-wait self-check: a barrier wait of at most `polls`
        polls that succeeds (complete=True) or runs out and raises the timeout
        bit in device_status() (complete=False).  Stream ordered."""
        L.check(L.lib().fftmv_check_bounded_wait(self.handle, int(polls), int(bool(complete)),
                                                 _stream_handle(stream, self.device)))

    # -- per-phase timers -----------------------------------------------------
    def set_timing(self, enable: bool = True) -> None:
        L.check(L.lib().fftmv_set_timing(self.handle, int(bool(enable))))

    def phase_times(self, which) -> tuple[list[float], int]:
        """Summed ms of [pad+FFT, block matvec, IFFT+unpad] and the call count."""
        ms = (ctypes.c_double * 3)()
        calls = ctypes.c_int64()
        L.check(L.lib().fftmv_phase_times(self.handle, _WHICH[which], ms, ctypes.byref(calls)))
        return list(ms), calls.value

    def reset_timing(self) -> None:
        L.check(L.lib().fftmv_reset_timing(self.handle))


# the C ABI's verbs, for callers that prefer functions
def set_precision(op: Operator, which, prec: str = "ddddd", mode: str = "native", fft_mode: str | None = None) -> None:
    op.set_precision(which, prec, mode, fft_mode)


def matvec(op: Operator, m, out=None, stream=None):
    return op.matvec(m, out=out, stream=stream)


def rmatvec(op: Operator, d, out=None, stream=None):
    return op.rmatvec(d, out=out, stream=stream)


def free(op: Operator) -> None:
    op.free()
