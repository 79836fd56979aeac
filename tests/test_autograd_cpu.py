"""CPU checks of the autograd wiring (no GPU): with the library's operator
replaced by the CPU oracle's F and F*, torch.autograd's numerical gradient
checks confirm that the backward of F m is F* g, the backward of F* d is F g,
and that second derivatives go through the same pair (Section 2.3: F* is the
adjoint F^T of the real operator).  tests/test_autograd.py runs the same
functions on the GPU operator."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2508_10202_gb300.autograd import ToeplitzLinear, toeplitz_matvec, toeplitz_rmatvec  # noqa: E402


class OracleOp:
    """matvec / rmatvec of the CPU oracle, in the operator's calling form."""

    def __init__(self, F):
        self.F = F
        self.calls = {"F": 0, "F*": 0}

    def matvec(self, m):
        self.calls["F"] += 1
        return torch.from_numpy(oracle.matvec_direct(self.F, m.detach().numpy()))

    def rmatvec(self, d):
        self.calls["F*"] += 1
        return torch.from_numpy(oracle.rmatvec_direct(self.F, d.detach().numpy()))


NT, ND, NM = 5, 3, 4


@pytest.fixture
def op():
    return OracleOp(synth.block_column(NT, ND, NM, seed=11))


@pytest.mark.parametrize("K", [None, 2])
def test_first_and_second_derivatives(op, K):
    shape_m = (NT, NM) if K is None else (K, NT, NM)
    shape_d = (NT, ND) if K is None else (K, NT, ND)
    g = torch.Generator().manual_seed(3)
    m = torch.randn(shape_m, dtype=torch.float64, generator=g, requires_grad=True)
    d = torch.randn(shape_d, dtype=torch.float64, generator=g, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: toeplitz_matvec(op, x), (m,))
    assert torch.autograd.gradcheck(lambda x: toeplitz_rmatvec(op, x), (d,))
    assert torch.autograd.gradgradcheck(lambda x: toeplitz_matvec(op, x), (m,))
    assert torch.autograd.gradgradcheck(lambda x: toeplitz_rmatvec(op, x), (d,))


def test_gradient_of_the_misfit_is_the_adjoint_residual(op):
    # L(m) = 1/2 ||F m - d||^2 has gradient F* (F m - d): one F forward, one F*
    # backward, no other operator calls
    g = torch.Generator().manual_seed(5)
    m = torch.randn((NT, NM), dtype=torch.float64, generator=g, requires_grad=True)
    d = torch.randn((NT, ND), dtype=torch.float64, generator=g)
    model = ToeplitzLinear(op)
    loss = 0.5 * (model(m) - d).pow(2).sum()
    loss.backward()
    assert op.calls == {"F": 1, "F*": 1}
    F = op.F
    want = oracle.rmatvec_direct(F, oracle.matvec_direct(F, m.detach().numpy()) - d.numpy())
    np.testing.assert_allclose(m.grad.numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
