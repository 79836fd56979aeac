"""Checkpoint of an operator's master F-hat (fftmv_get_fhat / fftmv_create_from_fhat,
Operator.save / Operator.load): the header format on the CPU, and on the GPU a
round trip whose operator gives bit-identical matvecs without a setup FFT."""
import numpy as np
import pytest

from paper_2508_10202_gb300.operator import FHAT_HEADER_BYTES, fhat_header, parse_fhat_header


def test_header_round_trip():
    h = fhat_header(1000, 100, 10000, 2000, 10000)
    assert len(h) == FHAT_HEADER_BYTES
    p = parse_fhat_header(h)
    assert (p["Nt"], p["Nd"], p["Nm"], p["L"], p["Nf"], p["ldn"]) == (1000, 100, 10000, 2000, 1001, 10000)


@pytest.mark.parametrize("block", [
    b"x" * FHAT_HEADER_BYTES,                                           # not JSON
    b'{"format": "other", "version": 1}'.ljust(FHAT_HEADER_BYTES),     # wrong format
    fhat_header(10, 2, 3, 20, 8)[:-1],                                  # short block
])
def test_header_rejects_other_files(block):
    with pytest.raises(ValueError):
        parse_fhat_header(block)


def test_header_rejects_inconsistent_sizes():
    import json
    good = json.loads(fhat_header(10, 2, 3, 20, 8).decode())
    for key, val in (("Nf", 12), ("ldn", 2), ("ldn", 12), ("L", 10), ("Nt", 0)):
        bad = dict(good, **{key: val})
        with pytest.raises(ValueError):
            parse_fhat_header(json.dumps(bad).encode().ljust(FHAT_HEADER_BYTES))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2508_10202_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("Nt,Nd,Nm", [(64, 8, 32), (50, 7, 99), (1000, 4, 9)])
def test_save_load_round_trip(torch_cuda, tmp_path, Nt, Nd, Nm):
    import synth
    from paper_2508_10202_gb300 import Operator
    torch = torch_cuda
    Fcol = synth.block_column(Nt, Nd, Nm, seed=7)
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, k=3, seed=8)).cuda()
    d = torch.from_numpy(synth.vectors(synth.TAG_D, Nt, Nd, k=3, seed=9)).cuda()
    a = Operator(torch.from_numpy(Fcol).cuda())
    path = tmp_path / "op.fhat"
    a.save(path)
    assert path.stat().st_size == FHAT_HEADER_BYTES + a.Nf * a.Nd * a.ldn * 16
    b = Operator.load(path)
    assert (b.Nt, b.Nd, b.Nm, b.L, b.ldn) == (a.Nt, a.Nd, a.Nm, a.L, a.ldn)
    for prec, mode, fft_mode in (("ddddd", "native", "native"), ("ddddd", "f64x2f32", "f64x2f32"),
                                 ("sssss", "native", "native"), ("sssss", "bf16x2", "native")):
        for op in (a, b):
            op.set_precision("F", prec, mode, fft_mode)
            op.set_precision("F*", prec, mode, fft_mode)
        x = (m, d) if prec == "ddddd" else (m.float(), d.float())
        ya, yb = a.matvec(x[0]).cpu().numpy(), b.matvec(x[0]).cpu().numpy()
        xa, xb = a.rmatvec(x[1]).cpu().numpy(), b.rmatvec(x[1]).cpu().numpy()
        assert np.array_equal(ya, yb) and np.array_equal(xa, xb), (prec, mode)
    # the same spectrum handed over in device memory
    fh = torch.empty(a.Nf * a.Nd * a.ldn * 2, dtype=torch.float64, device="cuda")
    from paper_2508_10202_gb300 import _lib as L
    L.check(L.lib().fftmv_get_fhat(a.handle, fh.data_ptr(), fh.numel() * 8, None))
    torch.cuda.synchronize()
    import ctypes
    h = ctypes.c_void_p()
    L.check(L.lib().fftmv_create_from_fhat(fh.data_ptr(), Nt, Nd, Nm, None, ctypes.byref(h)))
    c = Operator.__new__(Operator)
    c._attach(h)
    a.set_precision("F", "ddddd")
    c.set_precision("F", "ddddd")
    assert np.array_equal(a.matvec(m).cpu().numpy(), c.matvec(m).cpu().numpy())
    for op in (a, b, c):
        op.free()


@pytest.mark.gpu
def test_load_rejects_a_truncated_file(torch_cuda, tmp_path):
    import synth
    from paper_2508_10202_gb300 import Operator
    torch = torch_cuda
    a = Operator(torch.from_numpy(synth.block_column(16, 2, 3, seed=1)).cuda())
    path = tmp_path / "op.fhat"
    a.save(path)
    a.free()
    with open(path, "r+b") as f:
        f.truncate(FHAT_HEADER_BYTES + 100)
    with pytest.raises(ValueError):
        Operator.load(path)
