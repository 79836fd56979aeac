"""Seeded synthetic inputs for block lower-triangular Toeplitz matvecs.

This module is shared by the CPU oracle's tests and by the GPU library's tests
and benchmark, so that both sides see bit-identical inputs.  It holds random
draws, their scaling and the mantissa perturbation only: none of the matvec
arithmetic lives here.

Shapes follow the paper's notation (Section 2.3): the first block column of F
is a stack of Nt blocks F_k in R^{Nd x Nm} (lag k = 0..Nt-1, the paper's
F_{k+1,1}); a parameter vector m has Nt blocks m_j in R^{Nm}; a data vector d
has Nt blocks d_i in R^{Nd}.  Arrays are time-outer, space-inner:
``F[k, r, n]``, ``m[b, j, n]``, ``d[b, i, r]`` with b the right-hand side.

Every block is drawn from its own PCG64 stream keyed by
``SeedSequence([seed, tag, ...index])`` so that any block (a lag of the block
column, or one time block of one right-hand side) can be regenerated alone
and the result does not depend on how many threads drew it.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

TAG_BLOCK = 0   # block column F_k
TAG_M = 1       # parameter vectors m
TAG_D = 2       # data vectors d
TAG_NOISE = 3   # observation noise

__all__ = [
    "TAG_BLOCK", "TAG_M", "TAG_D", "TAG_NOISE",
    "block_generator", "block_column", "vectors", "perturb_mantissa",
]


def block_generator(seed: int, tag: int, *index: int) -> np.random.Generator:
    """The PCG64 generator that owns one block of one synthetic array."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(tag), *map(int, index)])))


def _threads(nbytes: int) -> int:
    if nbytes < (64 << 20):
        return 1
    return max(1, min(16, len(os.sched_getaffinity(0))))


def perturb_mantissa(x: np.ndarray) -> np.ndarray:
    """Set every FP64 fraction bit below the 23 leading ones to 1 (in place).

    Section 4.2.1: inputs are made not exactly representable in FP32 by setting
    the mantissa bits past position 23 to one; otherwise rounding to FP32 at
    the pad phase would cost nothing.  The 52-bit fraction keeps its leading
    23 bits; the trailing 29 bits become ones.  Zeros and non-finite values
    are left alone.  Returns ``x``.
    """
    if x.dtype != np.float64:
        raise TypeError("perturb_mantissa needs a float64 array")
    bits = x.view(np.uint64)
    finite_nonzero = np.isfinite(x) & (x != 0)
    low29 = np.uint64((1 << 29) - 1)
    np.bitwise_or(bits, low29, out=bits, where=finite_nonzero)
    return x


def block_column(Nt: int, Nd: int, Nm: int, seed: int = 0, decay: float | None = None,
                 dtype=np.float64, perturb: bool = False, out: np.ndarray | None = None) -> np.ndarray:
    """First block column F[k, r, n], k < Nt, entries iid N(0, 1).

    ``decay`` multiplies block k by exp(-k / decay) (the paper-shaped operator
    uses decay = 200 over the lag index).  ``perturb`` applies
    :func:`perturb_mantissa` after scaling.  Draws are FP64; ``dtype=float32``
    rounds them afterwards.
    """
    Nt, Nd, Nm = int(Nt), int(Nd), int(Nm)
    if out is None:
        out = np.empty((Nt, Nd, Nm), dtype=dtype)
    if out.shape != (Nt, Nd, Nm) or out.dtype != np.dtype(dtype):
        raise ValueError("out has the wrong shape or dtype")

    def fill(k: int) -> None:
        g = block_generator(seed, TAG_BLOCK, k)
        blk = g.standard_normal((Nd, Nm))
        if decay is not None:
            blk *= np.exp(-k / float(decay))
        if perturb:
            perturb_mantissa(blk)
        out[k] = blk

    nthreads = _threads(out.nbytes)
    if nthreads == 1:
        for k in range(Nt):
            fill(k)
    else:
        with ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(fill, range(Nt)))
    return out


def vectors(tag: int, Nt: int, N: int, k: int = 1, seed: int = 0, dtype=np.float64,
            perturb: bool = False, scale: float = 1.0) -> np.ndarray:
    """k stacked block vectors v[b, t, :] in R^N, t < Nt, entries iid N(0, scale^2).

    ``tag`` is TAG_M for parameter vectors (N = Nm), TAG_D for data vectors
    (N = Nd) and TAG_NOISE for noise.  Time block t of right-hand side b comes
    from the stream ``[seed, tag, b, t]``.
    """
    Nt, N, k = int(Nt), int(N), int(k)
    out = np.empty((k, Nt, N), dtype=dtype)

    def fill(bt: int) -> None:
        b, t = divmod(bt, Nt)
        g = block_generator(seed, tag, b, t)
        row = g.standard_normal(N)
        if scale != 1.0:
            row *= scale
        if perturb:
            perturb_mantissa(row)
        out[b, t] = row

    nthreads = _threads(out.nbytes)
    if nthreads == 1:
        for bt in range(k * Nt):
            fill(bt)
    else:
        with ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(fill, range(k * Nt), chunksize=64))
    return out
