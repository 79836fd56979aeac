"""GPU parity of the fused small-operator path (all five phases of Section 2.4
in one cluster launch, all FP64 or all FP32): against the CPU FP64 oracle and
against the three-kernel path of the same operator (fftmv_set_fusion)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5    # every phase in FP32 (the bar of the other FP32 tests)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


# (Nt, Nd, Nm, K): L = 128 or 256; channel counts from 1 to the 64 one cluster
# holds, odd ones, and both directions' widest side
CASES = [(64, 8, 32, 1), (64, 8, 32, 3), (64, 1, 1, 2), (64, 64, 64, 2), (128, 5, 37, 2), (127, 33, 2, 1),
         (61, 17, 64, 4), (128, 64, 1, 1), (64, 8, 32, 200)]   # the last: more clusters than fit at once


@pytest.mark.parametrize("Nt,Nd,Nm,K", CASES)
@pytest.mark.parametrize("io", [np.float64, np.float32])
@pytest.mark.parametrize("prec", ["ddddd", "sssss"])
def test_fused_matches_oracle_and_unfused(torch_cuda, Nt, Nd, Nm, K, io, prec):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Fcol = synth.block_column(Nt, Nd, Nm, seed=Nt + Nd)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=1).astype(io)
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=2).astype(io)
    op = Operator(torch.from_numpy(Fcol).cuda())
    assert op.info().L in (128, 256)
    op.set_precision("F", prec, "native", "native")
    op.set_precision("F*", prec, "native", "native")
    assert op.workspace_bytes("F", K) == 0 and op.workspace_bytes("F*", K) == 0   # no spectra in scratch
    mt, dt = torch.from_numpy(m).cuda(), torch.from_numpy(d).cuda()
    y = op.matvec(mt).cpu().numpy()
    x = op.rmatvec(dt).cpu().numpy()
    op.set_fusion(False)
    assert op.workspace_bytes("F", K) > 0
    y3 = op.matvec(mt).cpu().numpy()
    x3 = op.rmatvec(dt).cpu().numpy()
    assert op.device_status() == 0
    op.free()
    ref_d = oracle.matvec_direct(Fcol, m.astype(np.float64))
    ref_m = oracle.rmatvec_direct(Fcol, d.astype(np.float64))
    if prec == "ddddd":
        # FP64 throughout; FP32 I/O adds one rounding at the output; the two
        # paths are the same arithmetic up to the order of the FP64 sums
        tol = TOL64 if io == np.float64 else 2e-7
        tol3 = 1e-13 if io == np.float64 else 2e-7
    else:
        # FP32 throughout: both paths within the FP32 bar of the oracle, and
        # within it of each other (their FP32 sums run in different orders)
        tol = tol3 = TOL32
    for got, ref in ((y, ref_d), (x, ref_m), (y3, ref_d), (x3, ref_m)):
        assert np.all(np.isfinite(got))
        assert oracle.rel_l2(got, ref) <= tol
    assert oracle.rel_l2(y, y3) <= tol3
    assert oracle.rel_l2(x, x3) <= tol3


@pytest.mark.parametrize("prec,tol", [("ddddd", TOL64), ("sssss", TOL32)])
def test_fused_not_taken_outside_its_limits(torch_cuda, prec, tol):
    # 65 output channels (more than one cluster holds) and L = 200: the
    # three-kernel path, with its scratch
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    for Nt, Nd, Nm in ((64, 65, 8), (100, 4, 4)):
        Fcol = synth.block_column(Nt, Nd, Nm, seed=3)
        op = Operator(torch.from_numpy(Fcol).cuda())
        op.set_precision("F", prec, "native", "native")
        assert op.workspace_bytes("F", 1) > 0
        m = synth.vectors(synth.TAG_M, Nt, Nm, k=1, seed=4)
        y = op.matvec(torch.from_numpy(m).cuda()).cpu().numpy()
        assert oracle.rel_l2(y, oracle.matvec_direct(Fcol, m)) <= tol
        op.free()


@pytest.mark.parametrize("prec,mode,fft_mode", [("dssdd", "native", "native"), ("sssss", "bf16x2", "native"),
                                                ("ddddd", "f64x2f32", "native"), ("ddddd", "native", "f64x2f32")])
def test_fused_only_for_uniform_native_precision(torch_cuda, prec, mode, fft_mode):
    # mixed phases, the tensor cores and the double-float formats keep the
    # three-kernel path at a size the fused kernels take
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm = 64, 8, 32
    Fcol = synth.block_column(Nt, Nd, Nm, seed=5)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", prec, mode, fft_mode)
    assert op.workspace_bytes("F", 1) > 0
    op.set_precision("F", "sssss", "native", "f64x2f32")    # FP32 transforms: the FFT mode does not apply
    assert op.workspace_bytes("F", 1) == 0
    op.free()


@pytest.mark.parametrize("prec,tol", [("ddddd", TOL64), ("sssss", TOL32)])
def test_fused_in_a_cuda_graph_and_host_io(torch_cuda, prec, tol):
    # the fused launch replayed from a captured graph, and staged host I/O
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm = 64, 8, 32
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=1, seed=0)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", prec, "native", "native")
    assert op.workspace_bytes("F", 1) == 0
    ref = oracle.matvec_direct(Fcol, m)
    y_host = op.matvec(m)
    assert oracle.rel_l2(np.asarray(y_host), ref) <= tol
    s = torch.cuda.Stream()
    mt = torch.from_numpy(m).cuda()
    yt = torch.empty((1, Nt, Nd), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        op.matvec(mt, out=yt, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        op.matvec(mt, out=yt, stream=s)
    yt.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert oracle.rel_l2(yt.cpu().numpy(), ref) <= tol
    op.free()
