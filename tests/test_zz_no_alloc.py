"""The allocation-free entry point, fftmv_apply_noalloc, against fftmv_matvec/rmatvec.

fftmv_apply_noalloc serves callers that cannot allocate device memory once
they are running: for example a process whose memory manager reserved the
GPU's memory at start-up, or a latency-critical loop that must not risk an
allocation failing or a pool growing mid-run.  Its intermediate spectra live
in a fixed 64 MiB device array inside the library instead of the operator's
pool.  This test calls it through the C ABI twice in a row (the array keeps
the previous call's contents) and compares each result with the pooled entry
point's, within the tolerance of the other parity tests (FP64: 1e-12;
configurations with an FP32 phase: 1e-5), for the double-float and native
FP64 modes, the two tensor-core modes and FP32 I/O.  It lives in its own file,
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    from paper_2508_10202_gb300 import Operator, _lib
    return torch, Operator, _lib, _lib.lib()


def _noalloc(lib, op, which, x, out, stream):
    K = x.shape[0] if x.dim() == 3 else 1
    io = 0 if x.dtype.is_floating_point and x.element_size() == 8 else 1
    return lib.fftmv_apply_noalloc(op.handle, which, x.data_ptr(), out.data_ptr(), K, io, stream.cuda_stream)


@pytest.mark.parametrize("mode", ["native", "f64x2f32"])
def test_noalloc_matches_pooled_entry_points(env, mode):
    torch, Operator, L, lib = env
    Nt, Nd, Nm, K = 64, 8, 32, 3
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0)
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=0)).cuda()
    d = torch.from_numpy(synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=0)).cuda()
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", "ddddd", mode)
    op.set_precision("F*", "ddddd", mode)
    stream = torch.cuda.current_stream()
    ref_d = op.matvec(m).cpu().numpy()
    ref_m = op.rmatvec(d).cpu().numpy()
    for call in range(2):
        y = torch.full((K, Nt, Nd), float("nan"), dtype=torch.float64, device="cuda")
        x = torch.full((K, Nt, Nm), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, op, L.FFTMV_FORWARD, m, y, stream) == 0, lib.fftmv_last_error()
        assert _noalloc(lib, op, L.FFTMV_ADJOINT, d, x, stream) == 0, lib.fftmv_last_error()
        torch.cuda.synchronize()
        assert oracle.rel_l2(y.cpu().numpy(), ref_d) <= TOL64, call
        assert oracle.rel_l2(x.cpu().numpy(), ref_m) <= TOL64, call
    # and against the oracle itself
    assert oracle.rel_l2(y.cpu().numpy(), oracle.matvec_direct(Fcol, m.cpu().numpy())) <= TOL64
    op.free()


TOL32 = 1e-5   # configurations with an FP32 phase (tests/test_tensor.py)


@pytest.mark.parametrize("mode", ["bf16x2", "f16x2"])
@pytest.mark.parametrize("K", [3, 65])
@pytest.mark.parametrize("io", ["f64", "f32"])
def test_noalloc_tensor_core_modes(env, mode, K, io):
    # The tensor-core modes put more in the fixed array: the bf16/FP16 B planes
    # (cleared first when a chunk has padding rows: K = 3 pads each 6-row chunk
    # to 16, K = 65 leaves a one-RHS last chunk) and, for FP16, the per-RHS
    # maxima and scales behind them.  Each call must match the pooled call.
    torch, Operator, L, lib = env
    Nt, Nd, Nm = 64, 8, 32
    Fcol = synth.block_column(Nt, Nd, Nm, seed=2)
    dt = np.float64 if io == "f64" else np.float32
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=2).astype(dt)).cuda()
    d = torch.from_numpy(synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=2).astype(dt)).cuda()
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", "sssss", mode)
    op.set_precision("F*", "sssss", mode)
    stream = torch.cuda.current_stream()
    ref_d = op.matvec(m).double().cpu().numpy()
    ref_m = op.rmatvec(d).double().cpu().numpy()
    tdt = torch.float64 if io == "f64" else torch.float32
    for call in range(2):
        y = torch.full((K, Nt, Nd), float("nan"), dtype=tdt, device="cuda")
        x = torch.full((K, Nt, Nm), float("nan"), dtype=tdt, device="cuda")
        assert _noalloc(lib, op, L.FFTMV_FORWARD, m, y, stream) == 0, lib.fftmv_last_error()
        assert _noalloc(lib, op, L.FFTMV_ADJOINT, d, x, stream) == 0, lib.fftmv_last_error()
        torch.cuda.synchronize()
        assert oracle.rel_l2(y.double().cpu().numpy(), ref_d) <= TOL32, call
        assert oracle.rel_l2(x.double().cpu().numpy(), ref_m) <= TOL32, call
    assert oracle.rel_l2(y.double().cpu().numpy(), oracle.matvec_direct(Fcol, m.double().cpu().numpy())) <= TOL32
    assert op.device_status() == 0
    op.free()


def test_noalloc_fp32_io_double_float(env):
    # FP32 inputs and outputs through the FP64-class path
    torch, Operator, L, lib = env
    Nt, Nd, Nm, K = 64, 8, 32, 2
    Fcol = synth.block_column(Nt, Nd, Nm, seed=3)
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=3).astype(np.float32)).cuda()
    d = torch.from_numpy(synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=3).astype(np.float32)).cuda()
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", "ddddd", "f64x2f32")
    op.set_precision("F*", "ddddd", "f64x2f32")
    stream = torch.cuda.current_stream()
    ref_d = op.matvec(m).double().cpu().numpy()
    ref_m = op.rmatvec(d).double().cpu().numpy()
    for call in range(2):
        y = torch.full((K, Nt, Nd), float("nan"), dtype=torch.float32, device="cuda")
        x = torch.full((K, Nt, Nm), float("nan"), dtype=torch.float32, device="cuda")
        assert _noalloc(lib, op, L.FFTMV_FORWARD, m, y, stream) == 0, lib.fftmv_last_error()
        assert _noalloc(lib, op, L.FFTMV_ADJOINT, d, x, stream) == 0, lib.fftmv_last_error()
        torch.cuda.synchronize()
        assert oracle.rel_l2(y.double().cpu().numpy(), ref_d) <= TOL64, call
        assert oracle.rel_l2(x.double().cpu().numpy(), ref_m) <= TOL64, call
    op.free()


def test_noalloc_rejects_oversize_and_host_buffers(env):
    torch, Operator, L, lib = env
    Nt, Nd, Nm = 300, 4, 4000          # F needs Nf*ldn*16 = 301*4000*16 B per RHS
    op = Operator(torch.from_numpy(synth.block_column(Nt, Nd, Nm, seed=1)).cuda())
    K = 64                              # ~1.2 GB of spectra: beyond the fixed array
    need = op.workspace_bytes("F", K)
    assert need > 64 * 1024 * 1024
    m = torch.zeros((K, Nt, Nm), dtype=torch.float64, device="cuda")
    y = torch.zeros((K, Nt, Nd), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    assert _noalloc(lib, op, L.FFTMV_FORWARD, m, y, stream) == -3
    assert b"holds" in lib.fftmv_last_error()
    mh = np.zeros((Nt, Nm))
    yh = np.zeros((Nt, Nd))
    rc = lib.fftmv_apply_noalloc(op.handle, L.FFTMV_FORWARD, mh.ctypes.data, yh.ctypes.data, 1, 0,
                                 stream.cuda_stream)
    assert rc == -1 and b"device pointers" in lib.fftmv_last_error()
    op.free()


def test_noalloc_first_call_refused_inside_capture():
    # The first call on a device looks up the scratch array's address, which
    # must not happen inside a stream capture: in a fresh process, a first call
    # made while the stream is capturing returns FFTMV_ESTATE (-5) with a
    # message, the capture stays valid, and the same call succeeds afterwards.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r"""
import sys, torch
sys.path.insert(0, %r)
import synth
from paper_2508_10202_gb300 import Operator, build, _lib
build.build()
lib = _lib.lib()
op = Operator(torch.from_numpy(synth.block_column(16, 3, 8, seed=0)).cuda())
m = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
y = torch.empty((16, 3), dtype=torch.float64, device="cuda")
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.stream(s):
    g.capture_begin(capture_error_mode="thread_local")
    rc = lib.fftmv_apply_noalloc(op.handle, 0, m.data_ptr(), y.data_ptr(), 1, 0, s.cuda_stream)
    msg = lib.fftmv_last_error().decode()
    g.capture_end()
rc2 = lib.fftmv_apply_noalloc(op.handle, 0, m.data_ptr(), y.data_ptr(), 1, 0, s.cuda_stream)
torch.cuda.synchronize()
print(rc, rc2, "before capturing" in msg)
""" % root
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == "-5 0 True", r.stdout
