"""Failure detection without a GPU fault: every pipeline wait in the kernels is
bounded, and a wait that runs out raises FFTMV_STATUS_WAIT_TIMEOUT in the
operator's status word instead of hanging.  The self-check entry point makes
such a wait run out on purpose (a barrier that nothing completes, a small poll
limit) and the host reads the status; the context stays usable."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
def test_wait_that_runs_out_sets_the_status_and_the_context_stays_usable(torch_cuda):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300 import _lib as L
    Nt, Nd, Nm = 16, 3, 20
    Fcol = synth.block_column(Nt, Nd, Nm, seed=5)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=1, seed=5)
    op = Operator(torch.from_numpy(Fcol).cuda())
    assert op.device_status() == 0
    op.check_bounded_wait(polls=1000, complete=True)      # the phase completes: no bit
    assert op.device_status() == 0
    s = torch.cuda.Stream()
    op.check_bounded_wait(polls=1000, complete=False, stream=s)   # nothing completes it
    s.synchronize()
    assert op.device_status() == L.FFTMV_STATUS_WAIT_TIMEOUT
    assert op.device_status(clear=True) == L.FFTMV_STATUS_WAIT_TIMEOUT
    assert op.device_status() == 0
    # the same context still computes: a matvec afterwards matches the oracle
    y = op.matvec(torch.from_numpy(m).cuda()).cpu().numpy()
    ref = oracle.matvec_direct(Fcol, m)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    assert op.device_status() == 0
    for bad in (0, (1 << 22) + 1):
        with pytest.raises(L.FftmvError):
            op.check_bounded_wait(polls=bad)
    op.free()
