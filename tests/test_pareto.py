"""Pareto-front selection: host logic on CPU, the sweep on the GPU."""
import numpy as np
import pytest

from paper_2508_10202_gb300.pareto import CONFIGS, best_under, pareto_front


def test_front_and_selection_logic():
    pts = [{"prec": "a", "ms": 1.0, "rel_err": 1e-3}, {"prec": "b", "ms": 2.0, "rel_err": 1e-7},
           {"prec": "c", "ms": 1.5, "rel_err": 1e-2}, {"prec": "d", "ms": 3.0, "rel_err": 1e-15},
           {"prec": "e", "ms": 2.5, "rel_err": 1e-6}]
    front = pareto_front(pts)
    assert [p["prec"] for p in front] == ["a", "b", "d"]      # c and e are dominated
    assert best_under(pts, 1e-6)["prec"] == "b"
    assert best_under(pts, 1e-20) is None
    assert len(CONFIGS) == 32 and len(set(CONFIGS)) == 32


@pytest.mark.gpu
def test_sweep_on_gpu():
    import torch
    import oracle
    import synth
    from paper_2508_10202_gb300 import Operator, build
    from paper_2508_10202_gb300.pareto import sweep
    build.build()
    Nt, Nd, Nm = 100, 10, 400
    F = synth.block_column(Nt, Nd, Nm, seed=2, perturb=True)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=2, perturb=True)[0]
    op = Operator(torch.from_numpy(F).cuda())
    ref = torch.from_numpy(oracle.matvec_direct(F, m)).cuda()
    pts = sweep(op, "F", torch.from_numpy(m).cuda(), ref, reps=3)
    assert len(pts) == 60      # 28 configs with an FP64 FFT or block matvec x 2 modes + 4 without
    byname = {(p["prec"], p["mode"]): p for p in pts}
    assert byname[("ddddd", "native")]["rel_err"] <= 1e-12
    assert byname[("ddddd", "f64x2f32")]["rel_err"] <= 1e-12
    assert all(p["rel_err"] <= 1e-5 for p in pts)
    front = pareto_front(pts)
    assert front[-1]["rel_err"] <= 1e-12 and all(np.isfinite(p["ms"]) for p in front)
    op.free()
