"""Data-space Hessian assembly H_d = F G_prior F* + G_noise (Remark 1) against
the oracle's dense matrix A: H_d = prior_var A A^T + noise_var I."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("prec,mode,fft_mode,tol", [("ddddd", "f64x2f32", "f64x2f32", 1e-12),
                                                    ("sssss", "bf16x2", "native", 1e-5)])
def test_assemble_matches_dense(torch_cuda, prec, mode, fft_mode, tol):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.hessian import assemble
    Nt, Nd, Nm = 12, 3, 40
    Fcol = synth.block_column(Nt, Nd, Nm, seed=2)
    A = oracle.dense_matrix(Fcol)
    ref = 0.5 * A @ A.T + 0.01 * np.eye(Nt * Nd)
    op = Operator(torch.from_numpy(Fcol).cuda())
    for w in ("F", "F*"):
        op.set_precision(w, prec, mode, fft_mode)
    dt = torch.float64 if prec == "ddddd" else torch.float32
    H = assemble(op, prior_var=0.5, noise_var=0.01, batch=7, dtype=dt).double().cpu().numpy()
    assert np.linalg.norm(H - ref) <= tol * np.linalg.norm(ref)
    assert np.linalg.norm(H - H.T) <= 10 * tol * np.linalg.norm(ref)     # symmetric to rounding
    op.free()


def test_columns_subset_and_errors(torch_cuda):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.hessian import hessian_columns
    Nt, Nd, Nm = 9, 4, 17
    Fcol = synth.block_column(Nt, Nd, Nm, seed=3)
    A = oracle.dense_matrix(Fcol)
    op = Operator(torch.from_numpy(Fcol).cuda())
    for w in ("F", "F*"):
        op.set_precision(w, "ddddd", "f64x2f32", "f64x2f32")
    idx = [35, 0, 17, 17]
    cols = hessian_columns(op, idx, prior_var=2.0, batch=3).cpu().numpy().reshape(len(idx), -1)
    ref = 2.0 * (A @ A.T)[:, idx].T
    assert np.linalg.norm(cols - ref) <= 1e-12 * np.linalg.norm(ref)
    with pytest.raises(ValueError):
        hessian_columns(op, [Nt * Nd])
    op.free()


def test_columns_on_a_side_stream(torch_cuda):
    """With stream= given, building e_i, the two operator calls and the noise
    term all run on that stream; the result read after its synchronisation
    equals the default-stream one bit for bit."""
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.hessian import hessian_columns
    Nt, Nd, Nm = 40, 6, 300
    Fcol = synth.block_column(Nt, Nd, Nm, seed=4)
    op = Operator(torch.from_numpy(Fcol).cuda())
    for w in ("F", "F*"):
        op.set_precision(w, "ddddd", "f64x2f32", "f64x2f32")
    idx = list(range(0, Nt * Nd, 7))
    ref = hessian_columns(op, idx, prior_var=0.3, noise_var=0.02, batch=5)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    for handle in (s, s.cuda_stream):
        got = hessian_columns(op, idx, prior_var=0.3, noise_var=0.02, batch=5, stream=handle)
        s.synchronize()
        assert torch.equal(got, ref)
    op.free()
