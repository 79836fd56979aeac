"""GPU guard tests in place of a memory sanitizer: output buffers sit between
NaN-filled guard regions that must come back untouched (no write outside the
output), and caller scratch is NaN-filled before each call (no read of a
scratch entry the call did not write first: a NaN read would reach the
output)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GUARD = 4096   # elements on each side of the output


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


# (Nt, Nd, Nm, K, prec, mode, fft_mode, io): the fused small paths (FP64 and
# FP32), the three-kernel FP64 path, the double-float in-place FFTs
# (L = 2000), FP32, and the tensor cores with a ragged last chunk
CASES = [
    (64, 8, 32, 2, "ddddd", "native", "native", np.float64),
    (64, 8, 32, 2, "sssss", "native", "native", np.float64),
    (128, 33, 2, 3, "sssss", "native", "native", np.float32),
    (50, 7, 99, 3, "ddddd", "native", "native", np.float64),
    (1000, 4, 9, 2, "ddddd", "f64x2f32", "f64x2f32", np.float64),
    (1000, 4, 9, 2, "ddddd", "f64x2f32", "f64x2f32", np.float32),
    (256, 5, 37, 3, "sssss", "native", "native", np.float32),
    (128, 6, 70, 70, "sssss", "bf16x2", "native", np.float32),
    (100, 9, 40, 5, "sssss", "f16x2", "native", np.float32),
    # one right-hand side: the pipelined block matvecs, with ragged row
    # segments (Nd not a multiple of the rows per stage or per CTA) and
    # ragged column runs (a second, partial 512-pack run; a single short one)
    (64, 7, 99, 1, "ddddd", "f64x2f32", "f64x2f32", np.float64),
    (50, 5, 1300, 1, "sssss", "native", "native", np.float32),
    (1000, 3, 9, 1, "ddddd", "f64x2f32", "f64x2f32", np.float64),
    (128, 9, 600, 1, "ddddd", "f64x2f32", "f64x2f32", np.float32),
]


@pytest.mark.parametrize("Nt,Nd,Nm,K,prec,mode,fft_mode,io", CASES)
def test_outputs_stay_in_bounds_and_scratch_is_written_before_read(torch_cuda, Nt, Nd, Nm, K, prec, mode,
                                                                   fft_mode, io):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    tdt = torch.float64 if io == np.float64 else torch.float32
    Fcol = synth.block_column(Nt, Nd, Nm, seed=Nt + K)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=1).astype(io)
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=2).astype(io)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", prec, mode, fft_mode)
    op.set_precision("F*", prec, mode, fft_mode)
    tol = 1e-12 if prec == "ddddd" and io == np.float64 else 2e-7 if prec == "ddddd" else 1e-5
    for which, x, n_out, ref in (("F", m, Nd, oracle.matvec_direct), ("F*", d, Nm, oracle.rmatvec_direct)):
        n = K * Nt * n_out
        buf = torch.full((GUARD + n + GUARD,), float("nan"), dtype=tdt, device="cuda")
        out = buf[GUARD:GUARD + n].view(K, Nt, n_out)
        ws_bytes = op.workspace_bytes(which, K)
        ws = torch.full(((ws_bytes + 256 + 3) // 4,), float("nan"), dtype=torch.float32, device="cuda")
        wsb = ws.view(torch.uint8)
        off = (-wsb.data_ptr()) % 256
        op.apply_ws(which, torch.from_numpy(x).cuda(), out, wsb[off:off + ws_bytes])
        torch.cuda.synchronize()
        b = buf.cpu().numpy()
        assert np.all(np.isnan(b[:GUARD])) and np.all(np.isnan(b[GUARD + n:])), f"{which}: write outside the output"
        y = b[GUARD:GUARD + n].reshape(K, Nt, n_out)
        assert np.all(np.isfinite(y)), f"{which}: a NaN from unwritten scratch or a missed output"
        assert oracle.rel_l2(y, ref(Fcol, x.astype(np.float64))) <= tol
    assert op.device_status() == 0
    op.free()
