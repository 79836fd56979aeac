"""Data-space Hessian assembly, the many-right-hand-side workload of Remark 1.

Section 2 casts the operator as the parameter-to-observable map of a linear
Bayesian inverse problem with Gaussian prior N(m_prior, G_prior) and noise
N(0, G_noise); Remark 1 notes that sensor-placement studies re-assemble the
dense data-space matrix from Nd * Nt actions of F and F*.  The matrix built
here is

    H_d = F G_prior F* + G_noise        (Nt Nd x Nt Nd, data space)

with scalar (isotropic) G_prior = prior_var I and G_noise = noise_var I; its
column for data index i = t Nd + r is F(prior_var F*(e_i)) + noise_var e_i.
Columns go through the operator in batches: one rmatvec and one matvec of K
unit vectors each, so the tensor-core multi-RHS path serves the whole batch.
"""
from __future__ import annotations

import contextlib

__all__ = ["hessian_columns", "assemble"]


def hessian_columns(op, idx, prior_var: float = 1.0, noise_var: float = 0.0, batch: int = 64, dtype=None,
                    stream=None):
    """Columns idx (flat data indices t * Nd + r) of H_d as a (len(idx), Nt, Nd) tensor.

    The unit vectors are built on the device; the operator's current F and F*
    precision settings apply (FP32 / tensor cores for throughput, FP64-class
    for the ill-conditioned solves that follow).
    """
    import torch
    idx = torch.as_tensor(idx, dtype=torch.int64)
    n = op.Nt * op.Nd
    if idx.numel() and (int(idx.min()) < 0 or int(idx.max()) >= n):
        raise ValueError(f"data index out of range [0, {n})")
    if batch < 1:
        raise ValueError("batch must be >= 1")
    dtype = dtype or torch.float64
    dev = torch.device("cuda", op.device) if hasattr(op, "device") and isinstance(op.device, int) else "cuda"
    # every step (the torch ops building e_i and adding the noise, and the two
    # operator calls) is ordered on one stream
    if isinstance(stream, int):
        stream = torch.cuda.ExternalStream(stream)
    ctx = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with ctx:
        out = torch.empty((idx.numel(), op.Nt, op.Nd), dtype=dtype, device=dev)
        for c0 in range(0, idx.numel(), batch):
            ids = idx[c0:c0 + batch].to(dev)
            k = ids.numel()
            e = torch.zeros((k, op.Nt, op.Nd), dtype=dtype, device=dev)
            e.view(k, -1)[torch.arange(k, device=dev), ids] = 1.0
            x = op.rmatvec(e, stream=stream)
            if prior_var != 1.0:
                x.mul_(prior_var)
            y = op.matvec(x, stream=stream)
            if noise_var != 0.0:
                y.view(k, -1)[torch.arange(k, device=dev), ids] += noise_var
            out[c0:c0 + k] = y
    return out


def assemble(op, prior_var: float = 1.0, noise_var: float = 0.0, batch: int = 64, dtype=None):
    """The whole (Nt Nd) x (Nt Nd) matrix H_d, column by column (column i is row i: H_d is symmetric)."""
    import torch
    n = op.Nt * op.Nd
    cols = hessian_columns(op, torch.arange(n), prior_var, noise_var, batch, dtype)
    return cols.reshape(n, n).T.contiguous()
