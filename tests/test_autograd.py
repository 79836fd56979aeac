"""Autograd through the F / F* kernels (loss 1/2 ||F m - d||^2).

For the quadratic loss the gradient is F*(F m - d); its central finite
difference (L(m + h v) - L(m - h v)) / (2h) equals <grad, v> exactly in exact
arithmetic for every h, so in FP64 the check is limited by rounding only.
"""
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


def make_problem(Nt, Nd, Nm, seed):
    Fcol = synth.block_column(Nt, Nd, Nm, seed=seed)
    m_true = synth.vectors(synth.TAG_M, Nt, Nm, seed=seed)[0]
    return Fcol, m_true


def noisy_data(d_clean, Nt, Nd, seed):
    noise = synth.vectors(synth.TAG_NOISE, Nt, Nd, seed=seed)[0]
    return d_clean + 0.01 * np.linalg.norm(d_clean) / np.sqrt(Nt * Nd) * noise


def test_gradient_matches_oracle_and_finite_differences(torch_cuda):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.autograd import toeplitz_matvec
    Nt, Nd, Nm = 60, 12, 150
    Fcol, m_true = make_problem(Nt, Nd, Nm, seed=4)
    d = noisy_data(oracle.matvec_direct(Fcol, m_true), Nt, Nd, seed=4)
    m0 = synth.vectors(synth.TAG_M, Nt, Nm, seed=5)[0]
    g_ref = oracle.rmatvec_direct(Fcol, oracle.matvec_direct(Fcol, m0) - d)
    op = Operator(torch.from_numpy(Fcol).cuda())

    # FP32 compute: gradient within the FP32 tolerance of the oracle gradient
    op.set_precision("F", "sssss")
    op.set_precision("F*", "sssss")
    m = torch.tensor(m0, dtype=torch.float32, device="cuda", requires_grad=True)
    dt = torch.tensor(d, dtype=torch.float32, device="cuda")
    loss = 0.5 * ((toeplitz_matvec(op, m) - dt) ** 2).sum()
    loss.backward()
    assert oracle.rel_l2(m.grad.double().cpu().numpy(), g_ref) <= 1e-5

    # FP64 (FP64-class kernels): oracle gradient and 16 finite-difference directions
    op.set_precision("F", "ddddd", "f64x2f32")
    op.set_precision("F*", "ddddd", "f64x2f32")
    m = torch.tensor(m0, dtype=torch.float64, device="cuda", requires_grad=True)
    dt = torch.tensor(d, dtype=torch.float64, device="cuda")

    def L(x):
        return 0.5 * ((toeplitz_matvec(op, x) - dt) ** 2).sum()

    L(m).backward()
    g = m.grad.detach()
    assert oracle.rel_l2(g.cpu().numpy(), g_ref) <= 1e-12
    rng = np.random.default_rng(6)
    with torch.no_grad():
        for _ in range(16):
            v = torch.tensor(rng.standard_normal((Nt, Nm)), device="cuda")
            h = 1e-3 * m.norm() / v.norm()
            fd = (L(m + h * v) - L(m - h * v)) / (2 * h)
            gv = (g * v).sum()
            assert abs(fd - gv) <= 1e-8 * abs(gv) + 1e-10 * g.norm() * v.norm()
    op.free()


def test_double_backward_is_forward(torch_cuda):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.autograd import ToeplitzLinear, toeplitz_rmatvec
    Nt, Nd, Nm = 20, 5, 30
    Fcol, _ = make_problem(Nt, Nd, Nm, seed=9)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", "ddddd", "f64x2f32")
    op.set_precision("F*", "ddddd", "f64x2f32")
    u = torch.tensor(synth.vectors(synth.TAG_M, Nt, Nm, seed=1)[0], device="cuda")
    d = torch.tensor(synth.vectors(synth.TAG_D, Nt, Nd, seed=1)[0], device="cuda", requires_grad=True)
    (toeplitz_rmatvec(op, d) * u).sum().backward()           # d/dd <F* d, u> = F u
    assert oracle.rel_l2(d.grad.cpu().numpy(), oracle.matvec_direct(Fcol, u.cpu().numpy())) <= 1e-12
    # Hessian-vector product of 1/2 ||F x||^2 through double backward: F* F v
    layer = ToeplitzLinear(op)
    x = u.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(0.5 * (layer(x) ** 2).sum(), x, create_graph=True)
    v = torch.tensor(synth.vectors(synth.TAG_M, Nt, Nm, seed=2)[0], device="cuda")
    (hv,) = torch.autograd.grad((g * v).sum(), x)
    ref = oracle.rmatvec_direct(Fcol, oracle.matvec_direct(Fcol, v.cpu().numpy()))
    assert oracle.rel_l2(hv.cpu().numpy(), ref) <= 1e-12
    op.free()


@pytest.mark.slow
def test_fullsize_differentiable_adjoint(torch_cuda):
    """Nt=500, Nd=200, Nm=5000, FP32 compute; 1% noise; FD on 16 directions in FP64."""
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.autograd import toeplitz_matvec
    Nt, Nd, Nm = 500, 200, 5000
    Fcol, m_true = make_problem(Nt, Nd, Nm, seed=0)
    op = Operator(Fcol)
    op.set_precision("F", "ddddd", "f64x2f32")
    op.set_precision("F*", "ddddd", "f64x2f32")
    mt = torch.tensor(m_true, device="cuda")
    d_clean = op.matvec(mt).cpu().numpy()
    d = torch.tensor(noisy_data(d_clean, Nt, Nd, seed=0), device="cuda")
    m0 = torch.tensor(synth.vectors(synth.TAG_M, Nt, Nm, seed=1)[0], device="cuda")

    def grad_at(dtype):
        m = m0.to(dtype).clone().requires_grad_(True)
        loss = 0.5 * ((toeplitz_matvec(op, m) - d.to(dtype)) ** 2).sum()
        loss.backward()
        return m.grad.double()

    g64 = grad_at(torch.float64)
    # sampled entries of the FP64-class gradient against the oracle's F* of the same residual
    res = (op.matvec(m0) - d).cpu().numpy()
    rng = np.random.default_rng(2)
    idx = [(int(rng.integers(Nt)), int(rng.integers(Nm))) for _ in range(30)]
    ref = oracle.rmatvec_entries(Fcol, res, idx)
    got = np.array([g64[j, n].item() for j, n in idx])
    assert oracle.rel_l2(got, ref) <= 1e-12
    # FP32 compute against FP64
    op.set_precision("F", "sssss")
    op.set_precision("F*", "sssss")
    g32 = grad_at(torch.float32)
    assert float((g32 - g64).norm() / g64.norm()) <= 1e-5
    # finite differences in FP64
    op.set_precision("F", "ddddd", "f64x2f32")
    op.set_precision("F*", "ddddd", "f64x2f32")
    rng = np.random.default_rng(3)
    with torch.no_grad():
        def L(x):
            return 0.5 * ((op.matvec(x) - d) ** 2).sum()
        for _ in range(16):
            v = torch.tensor(rng.standard_normal((Nt, Nm)), device="cuda")
            h = 1e-3 * m0.norm() / v.norm()
            fd = (L(m0 + h * v) - L(m0 - h * v)) / (2 * h)
            gv = (g64 * v).sum()
            assert abs(fd - gv) <= 1e-8 * abs(gv) + 1e-10 * g64.norm() * v.norm()
    op.free()
