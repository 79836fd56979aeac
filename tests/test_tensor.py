"""GPU parity of the multi-right-hand-side tensor-core path (gemv_mode BF16X2).

F-hat and the transformed inputs are split into bfloat16 hi + lo parts and
multiplied on the tcgen05 tensor cores with FP32 accumulation, so the result
is at FP32 level: relative L2 <= 1e-5 against the FP64 oracle, the tolerance
for configurations with an FP32 phase.  The cases cover one and several
right-hand-side chunks (64 per chunk, a short last chunk), one and two 128-row
M tiles (Nd > 128), odd channel counts and every FFT length family.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
CASES = [  # Nt, Nd, Nm, K
    (64, 8, 32, 1),
    (40, 13, 300, 5),
    (25, 3, 77, 16),
    (64, 100, 1000, 64),
    (30, 130, 200, 16),
    (20, 7, 99, 70),
    (125, 64, 513, 33),
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("Nt,Nd,Nm,K", CASES)
@pytest.mark.parametrize("prec", ["sssss", "ddsdd"])
@pytest.mark.parametrize("mode", ["bf16x2", "f16x2"])
def test_tensor_core_forward(torch_cuda, Nt, Nd, Nm, K, prec, mode, record_property):
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    seed = Nt + Nd + Nm + K
    Fcol = synth.block_column(Nt, Nd, Nm, seed=seed)
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=seed)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", prec, mode)
    y = op.matvec(torch.from_numpy(m).cuda()).cpu().numpy()
    ref = oracle.matvec_direct(Fcol, m)
    err = oracle.rel_l2(y, ref)
    record_property("rel_l2", err)
    assert err <= TOL, err
    # per right-hand side too: no chunk or column is off
    for b in range(K):
        assert oracle.rel_l2(y[b], ref[b]) <= 3 * TOL, b
    assert op.device_status() == 0
    # FP32 I/O through the same path
    y32 = op.matvec(torch.from_numpy(m.astype(np.float32)).cuda()).cpu().numpy()
    assert oracle.rel_l2(y32, oracle.matvec_direct(Fcol, m.astype(np.float32).astype(np.float64))) <= TOL
    op.free()


@pytest.mark.parametrize("Nt,Nd,Nm,K", CASES + [(30, 200, 1000, 9), (16, 8, 300, 1)])
@pytest.mark.parametrize("prec", ["sssss", "ddsdd"])
@pytest.mark.parametrize("mode", ["bf16x2", "f16x2"])
def test_tensor_core_adjoint(torch_cuda, Nt, Nd, Nm, K, prec, mode):
    # F* on the tensor cores: F-hat read transposed (MN-major), conjugate in the epilogue
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    seed = 3 * Nt + Nd + Nm + K
    Fcol = synth.block_column(Nt, Nd, Nm, seed=seed)
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=seed)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F*", prec, mode)
    x = op.rmatvec(torch.from_numpy(d).cuda()).cpu().numpy()
    ref = oracle.rmatvec_direct(Fcol, d)
    assert oracle.rel_l2(x, ref) <= TOL
    for b in range(K):
        assert oracle.rel_l2(x[b], ref[b]) <= 3 * TOL, b
    assert op.device_status() == 0
    op.free()


def test_tensor_core_mode_rules(torch_cuda):
    torch = torch_cuda
    from paper_2508_10202_gb300 import FftmvError, Operator
    Fcol = synth.block_column(8, 2, 16, seed=3)
    op = Operator(torch.from_numpy(Fcol).cuda())
    with pytest.raises(FftmvError, match="FP32 GEMV"):
        op.set_precision("F", "ddddd", "bf16x2")
    with pytest.raises(FftmvError, match="FP32 GEMV"):
        op.set_precision("F*", "ddddd", "f16x2")
    op.set_precision("F*", "sssss", "bf16x2")
    op.set_precision("F", "sssss", "f16x2")
    op.free()


def test_tensor_core_matches_cuda_core_fp32(torch_cuda):
    # the same operator through the FP32 CUDA-core matvec and the tensor cores
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Fcol = synth.block_column(50, 20, 400, seed=8)
    m = torch.from_numpy(synth.vectors(synth.TAG_M, 50, 400, k=12, seed=8)).cuda()
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision("F", "sssss", "native")
    a = op.matvec(m).cpu().numpy()
    op.set_precision("F", "sssss", "bf16x2")
    b = op.matvec(m).cpu().numpy()
    assert oracle.rel_l2(b, a) <= 2 * TOL
    op.free()


@pytest.mark.parametrize("which", ["F", "F*"])
@pytest.mark.parametrize("mode", ["bf16x2", "f16x2"])
def test_tensor_core_many_tiles_per_cta(torch_cuda, which, mode):
    # F: 301 frequencies (two tiles for some of the 152 persistent CTAs); F*: 301 x 5
    # M tiles (about ten each): the pipeline phases carry across tiles.  Checked
    # against the oracle's FFT path (pinned to the definition in test_oracle.py).
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm, K = 300, 100, 640, 64
    Fcol = synth.block_column(Nt, Nd, Nm, seed=41)
    op = Operator(torch.from_numpy(Fcol).cuda())
    op.set_precision(which, "sssss", mode)
    if which == "F":
        x = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=41)
        got = op.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = oracle.matvec_fft(Fcol, x)
    else:
        x = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=41)
        got = op.rmatvec(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = oracle.rmatvec_fft(Fcol, x)
    assert oracle.rel_l2(got, ref) <= TOL
    for b in (0, 31, 63):
        assert oracle.rel_l2(got[b], ref[b]) <= 3 * TOL
    assert op.device_status() == 0
    op.free()


@pytest.mark.parametrize("fscale,xscale", [(1e6, 1e-5), (1e-6, 1e7), (1.0, 1.0)])
def test_fp16_scaling_covers_the_range(torch_cuda, fscale, xscale, record_property):
    # FP16 alone spans 6e-5 .. 65504: the per-frequency and per-RHS powers of two
    # keep F-hat and the spectra inside it whatever their magnitudes
    torch = torch_cuda
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm, K = 50, 12, 300, 8
    Fcol = synth.block_column(Nt, Nd, Nm, seed=51) * fscale
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=K, seed=51) * xscale
    m[3] *= 1e-3                                  # right-hand sides of different sizes in one call
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=K, seed=51) * xscale
    op = Operator(torch.from_numpy(Fcol).cuda())
    errs = {}
    for mode in ("bf16x2", "f16x2"):
        op.set_precision("F", "sssss", mode)
        op.set_precision("F*", "sssss", mode)
        y = op.matvec(torch.from_numpy(m).cuda()).cpu().numpy()
        x = op.rmatvec(torch.from_numpy(d).cuda()).cpu().numpy()
        ry, rx = oracle.matvec_direct(Fcol, m), oracle.rmatvec_direct(Fcol, d)
        errs[mode] = (max(oracle.rel_l2(y[b], ry[b]) for b in range(K)), oracle.rel_l2(x, rx))
        assert errs[mode][0] <= 3 * TOL and errs[mode][1] <= TOL, (mode, errs[mode])
        assert np.isfinite(y).all() and np.isfinite(x).all()
    record_property("errors", errs)
    op.free()
