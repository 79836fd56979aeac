"""GPU parity of the fused small-operator path (all five phases of Section 2.4
in one cluster launch, all FP64): against the CPU FP64 oracle and against the
three-kernel path of the same operator (fftmv_set_fusion)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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
def test_fused_matches_oracle_and_unfused(torch_cuda, Nt, Nd, Nm, K, io):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Fcol = synth.block_column(Nt, Nd, Nm, seed=Nt + Nd)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=1).astype(io)
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=2).astype(io)
    op = Operator(torch.from_numpy(Fcol).cuda())
    assert op.info().L in (128, 256)
    op.set_precision("F", "ddddd", "native", "native")
    op.set_precision("F*", "ddddd", "native", "native")
    assert op.workspace_bytes("F", K) == 0 and op.workspace_bytes("F*", K) == 0   # no spectra in scratch
    mt, dt = torch.from_numpy(m).cuda(), torch.from_numpy(d).cuda()
    y = op.matvec(mt).cpu().numpy()
    x = op.rmatvec(dt).cpu().numpy()
    op.set_fusion(False)
    assert op.workspace_bytes("F", K) > 0
    y3 = op.matvec(mt).cpu().numpy()
    x3 = op.rmatvec(dt).cpu().numpy()
    op.free()
    # FP64 throughout; FP32 I/O adds one rounding at the output
    tol = TOL64 if io == np.float64 else 2e-7
    assert oracle.rel_l2(y, oracle.matvec_direct(Fcol, m.astype(np.float64))) <= tol
    assert oracle.rel_l2(x, oracle.rmatvec_direct(Fcol, d.astype(np.float64))) <= tol
    # the same arithmetic up to the order of the FP64 sums
    assert oracle.rel_l2(y, y3) <= (1e-13 if io == np.float64 else 2e-7)
    assert oracle.rel_l2(x, x3) <= (1e-13 if io == np.float64 else 2e-7)


def test_fused_not_taken_outside_its_limits(torch_cuda):
    # 65 output channels (more than one cluster holds) and L = 200: the
    # three-kernel path, with its scratch
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    for Nt, Nd, Nm in ((64, 65, 8), (100, 4, 4)):
        Fcol = synth.block_column(Nt, Nd, Nm, seed=3)
        op = Operator(torch.from_numpy(Fcol).cuda())
        op.set_precision("F", "ddddd", "native", "native")
        assert op.workspace_bytes("F", 1) > 0
        m = synth.vectors(synth.TAG_M, Nt, Nm, k=1, seed=4)
        y = op.matvec(torch.from_numpy(m).cuda()).cpu().numpy()
        assert oracle.rel_l2(y, oracle.matvec_direct(Fcol, m)) <= TOL64
        op.free()


def test_fused_in_a_cuda_graph_and_host_io(torch_cuda):
    # the fused launch replayed from a captured graph, and staged host I/O
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm = 64, 8, 32
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=1, seed=0)
    op = Operator(torch.from_numpy(Fcol).cuda())
    ref = oracle.matvec_direct(Fcol, m)
    y_host = op.matvec(m)
    assert oracle.rel_l2(np.asarray(y_host), ref) <= TOL64
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
    assert oracle.rel_l2(yt.cpu().numpy(), ref) <= TOL64
    op.free()
