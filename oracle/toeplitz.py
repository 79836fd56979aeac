"""CPU oracle for block lower-triangular Toeplitz matvecs (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the graft
entry point and the benchmark's CPU-baseline / reference leg may import this
package.  The GPU library never calls it, and it shares no code with the GPU
library: its inputs come from the ``synth`` generators or from the caller.

Notation (Section 2.3 of the paper, Eq. (ShiftInvariance)): F has Nt x Nt
blocks, each Nd x Nm; only the first block column F_k = F_{k+1,1}
(k = 0..Nt-1, 0-based lag) is stored.  Arrays are time-outer:
``Fcol[k, r, n]``, ``m[j, n]``, ``d[i, r]``; a leading axis stacks right-hand
sides.

Functions, each a plain restatement of one passage:

* :func:`matvec_direct`, :func:`rmatvec_direct` - the definition of F and of
  its adjoint (Section 2.3): d_i = sum_{j<=i} F_{i-j} m_j and
  m*_j = sum_{i>=j} F_{i-j}^T d_i.  Primary oracle.
* :func:`dense_matrix` - the block matrix of Section 2.3 assembled entry by
  entry (brute force for tiny sizes).
* :func:`spectrum`, :func:`matvec_fft`, :func:`rmatvec_fft` - the five phases
  of the matvec algorithm (Section 2.4): zero pad to 2Nt, FFT along time,
  per-frequency block matvec (conjugate transpose for F*), inverse FFT, unpad.
* :func:`matvec_mixed`, :func:`rmatvec_mixed` - the same five phases with each
  phase computed in FP32 or FP64 as a precision string names (Section 3.2).
* :func:`matvec_entries`, :func:`rmatvec_entries` - selected outputs of the
  definition, one at a time, for full-size spot checks.
* :func:`relative_error_bound`, :func:`error_bound` - the first-order bound
  of Eq. (error), Section 3.2.1, with all algorithm constants set to one;
  the second picks n_m and p_c (F) or n_d and p_r (F*) from the grid.
* :func:`hessian_entries` - entries of the data-space Hessian
  F G_prior F* + G_noise of Remark 1 (isotropic G_prior and G_noise), each
  from the definition as an inner product of two block rows of F.

Pins (tests/test_oracle.py) tie these to closed forms, brute force, the
adjoint identity, causality and the spectrum facts; nothing here is compared
only against itself.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

__all__ = [
    "matvec_direct", "rmatvec_direct", "dense_matrix",
    "spectrum", "matvec_fft", "rmatvec_fft", "matvec_fft_spec", "rmatvec_fft_spec",
    "matvec_mixed", "rmatvec_mixed", "parse_precision",
    "matvec_entries", "rmatvec_entries", "relative_error_bound", "error_bound", "rel_l2",
    "hessian_entries",
]


def _stack(x: np.ndarray, ndim: int) -> tuple[np.ndarray, bool]:
    """Add a right-hand-side axis if ``x`` has none."""
    if x.ndim == ndim:
        return x[None], True
    if x.ndim == ndim + 1:
        return x, False
    raise ValueError(f"expected {ndim} or {ndim + 1} dimensions, got {x.ndim}")


def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error ||x - ref|| / ||ref|| over the whole array, in FP64."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((x - ref).ravel())
    return float(num / den) if den > 0 else float(num)


# ---------------------------------------------------------------------------
# The definition (Section 2.3)
# ---------------------------------------------------------------------------

def matvec_direct(Fcol: np.ndarray, m: np.ndarray) -> np.ndarray:
    """d = F m from the block lower-triangular Toeplitz definition.

    Section 2.3, Eq. (ShiftInvariance): block (i, j) of F is F_{i-j} for
    j <= i and 0 above the diagonal, so d_i = sum_{j=0}^{i} F_{i-j} m_j.
    Summed by lag k = i - j: every output block i >= k receives F_k m_{i-k}.
    ``m`` is [Nt, Nm] or [K, Nt, Nm]; the result is [Nt, Nd] or [K, Nt, Nd].
    """
    Fcol = np.asarray(Fcol, dtype=np.float64)
    Nt, Nd, Nm = Fcol.shape
    mm, squeeze = _stack(np.asarray(m, dtype=np.float64), 2)
    if mm.shape[1:] != (Nt, Nm):
        raise ValueError("m does not match the block column")
    d = np.zeros((mm.shape[0], Nt, Nd))
    for k in range(Nt):
        # d[:, i, :] += F_k @ m[:, i - k, :] for i = k .. Nt-1
        d[:, k:, :] += mm[:, : Nt - k, :] @ Fcol[k].T
    return d[0] if squeeze else d


def rmatvec_direct(Fcol: np.ndarray, d: np.ndarray) -> np.ndarray:
    """m* = F* d, the adjoint of :func:`matvec_direct` (Euclidean inner products).

    F is real, so F* = F^T: block (j, i) of F^T is F_{i-j}^T for i >= j, and
    m*_j = sum_{i=j}^{Nt-1} F_{i-j}^T d_i (Section 2.3; Section 2.4 states F*
    runs the same phases with the conjugate-transpose block matvec).
    """
    Fcol = np.asarray(Fcol, dtype=np.float64)
    Nt, Nd, Nm = Fcol.shape
    dd, squeeze = _stack(np.asarray(d, dtype=np.float64), 2)
    if dd.shape[1:] != (Nt, Nd):
        raise ValueError("d does not match the block column")
    ms = np.zeros((dd.shape[0], Nt, Nm))
    for k in range(Nt):
        # m*[:, j, :] += F_k^T d[:, j + k, :] for j = 0 .. Nt-1-k
        ms[:, : Nt - k, :] += dd[:, k:, :] @ Fcol[k]
    return ms[0] if squeeze else ms


def dense_matrix(Fcol: np.ndarray) -> np.ndarray:
    """The full (Nt*Nd) x (Nt*Nm) matrix of Section 2.3, entry by entry.

    Row index i*Nd + r, column index j*Nm + n; entry F_{i-j}[r, n] when
    j <= i, else 0.  Pure loops: tiny sizes only.
    """
    Fcol = np.asarray(Fcol, dtype=np.float64)
    Nt, Nd, Nm = Fcol.shape
    A = np.zeros((Nt * Nd, Nt * Nm))
    for i in range(Nt):
        for j in range(Nt):
            if j > i:
                continue
            for r in range(Nd):
                for n in range(Nm):
                    A[i * Nd + r, j * Nm + n] = Fcol[i - j, r, n]
    return A


# ---------------------------------------------------------------------------
# The five-phase FFT algorithm (Section 2.4)
# ---------------------------------------------------------------------------

def spectrum(Fcol: np.ndarray, L: int | None = None) -> np.ndarray:
    """Setup: F-hat = FFT along time of the zero-padded first block column.

    Section 2.4: F embeds in a block circulant matrix by zero padding its first
    block column to length L = 2 Nt; the DFT block-diagonalises it.  Returns
    F-hat[w, r, n] = sum_{k<Nt} F_k[r, n] exp(-2 pi i w k / L) for
    w = 0 .. L/2 (the half spectrum of a real signal), complex128.
    """
    Fcol = np.asarray(Fcol, dtype=np.float64)
    Nt = Fcol.shape[0]
    L = 2 * Nt if L is None else int(L)
    return scipy.fft.rfft(Fcol, n=L, axis=0)


def matvec_fft_spec(Fhat: np.ndarray, m: np.ndarray, Nt: int, L: int | None = None) -> np.ndarray:
    """Phases 1-5 of Section 2.4 for F, given the setup spectrum F-hat.

    1. zero pad each channel of m in time from Nt to L (= 2 Nt);
    2. m-hat = FFT along time (half spectrum, w = 0..L/2);
    3. d-hat_w = F-hat_w m-hat_w for every frequency (batched block matvec);
    4. d = inverse FFT along time;
    5. keep the first Nt time samples (unpad).
    """
    L = 2 * Nt if L is None else int(L)
    mm, squeeze = _stack(np.asarray(m, dtype=np.float64), 2)
    m_pad = np.zeros((mm.shape[0], L, mm.shape[2]))
    m_pad[:, :Nt, :] = mm                                       # phase 1
    m_hat = scipy.fft.rfft(m_pad, axis=1)                       # phase 2: [K, Nf, Nm]
    d_hat = np.matmul(Fhat[None], m_hat[..., None])[..., 0]     # phase 3: [K, Nf, Nd]
    d_full = scipy.fft.irfft(d_hat, n=L, axis=1)                # phase 4
    d = d_full[:, :Nt, :]                                       # phase 5
    return d[0] if squeeze else d


def rmatvec_fft_spec(Fhat: np.ndarray, d: np.ndarray, Nt: int, L: int | None = None) -> np.ndarray:
    """Phases 1-5 of Section 2.4 for F*: phase 3 uses the conjugate transpose.

    m*-hat_w = F-hat_w^H d-hat_w.  Zero padding d at the end of time makes the
    circulant's transpose agree with the block upper-triangular F^T on the
    first Nt output blocks.
    """
    L = 2 * Nt if L is None else int(L)
    dd, squeeze = _stack(np.asarray(d, dtype=np.float64), 2)
    d_pad = np.zeros((dd.shape[0], L, dd.shape[2]))
    d_pad[:, :Nt, :] = dd
    d_hat = scipy.fft.rfft(d_pad, axis=1)
    m_hat = np.matmul(np.conj(Fhat).transpose(0, 2, 1)[None], d_hat[..., None])[..., 0]
    m_full = scipy.fft.irfft(m_hat, n=L, axis=1)
    ms = m_full[:, :Nt, :]
    return ms[0] if squeeze else ms


def matvec_fft(Fcol: np.ndarray, m: np.ndarray, L: int | None = None) -> np.ndarray:
    """F m by the FFT algorithm of Section 2.4 (setup included)."""
    Nt = np.asarray(Fcol).shape[0]
    return matvec_fft_spec(spectrum(Fcol, L), m, Nt, L)


def rmatvec_fft(Fcol: np.ndarray, d: np.ndarray, L: int | None = None) -> np.ndarray:
    """F* d by the FFT algorithm of Section 2.4 (setup included)."""
    Nt = np.asarray(Fcol).shape[0]
    return rmatvec_fft_spec(spectrum(Fcol, L), d, Nt, L)


# ---------------------------------------------------------------------------
# Per-phase mixed precision (Section 3.2)
# ---------------------------------------------------------------------------

PHASES = ("pad", "fft", "gemv", "ifft", "unpad")


def parse_precision(prec: str) -> tuple[np.dtype, ...]:
    """A 5-letter string over {d, s}: one letter per phase in execution order.

    Section 3.2: each of the five phases (pad, FFT, block matvec, IFFT, unpad)
    runs in single or double precision, 32 configurations in all.  'd' means
    FP64, 's' FP32.
    """
    if len(prec) != 5 or any(c not in "ds" for c in prec):
        raise ValueError(f"precision string must be 5 letters over d/s, got {prec!r}")
    return tuple(np.dtype(np.float64) if c == "d" else np.dtype(np.float32) for c in prec)


def _complex_of(real: np.dtype) -> np.dtype:
    return np.dtype(np.complex128) if real == np.float64 else np.dtype(np.complex64)


def _mixed(Fhat: np.ndarray, x: np.ndarray, Nt: int, prec: str, adjoint: bool) -> np.ndarray:
    """Shared body of :func:`matvec_mixed` / :func:`rmatvec_mixed`.

    Section 3.2: input and output are FP64; every phase computes in its own
    precision and its input is cast to that precision on entry (a cast that
    rounds when the precision drops, exact when it rises); the matrix F-hat is
    held in the block-matvec phase's precision; the setup spectrum is FP64.
    The memory-only reorders between phases run at the lower of the two
    neighbouring precisions, which the casts on entry already reproduce.
    """
    p_pad, p_fft, p_gemv, p_ifft, p_unpad = parse_precision(prec)
    L = 2 * Nt
    xx, squeeze = _stack(np.asarray(x, dtype=np.float64), 2)
    K, _, N_in = xx.shape
    # phase 1: zero pad (and broadcast, a no-op on one device), in p_pad
    v1 = np.zeros((K, L, N_in), dtype=p_pad)
    v1[:, :Nt, :] = xx.astype(p_pad)
    # phase 2: FFT along time in p_fft
    v2 = scipy.fft.rfft(v1.astype(p_fft), axis=1)
    assert v2.dtype == _complex_of(p_fft)
    # phase 3: block-diagonal matvec in p_gemv, F-hat stored in p_gemv
    cg = _complex_of(p_gemv)
    Fg = Fhat.astype(cg)
    v2g = v2.astype(cg)
    if adjoint:
        v3 = np.matmul(np.conj(Fg).transpose(0, 2, 1)[None], v2g[..., None])[..., 0]
    else:
        v3 = np.matmul(Fg[None], v2g[..., None])[..., 0]
    assert v3.dtype == cg
    # phase 4: inverse FFT in p_ifft
    v4 = scipy.fft.irfft(v3.astype(_complex_of(p_ifft)), n=L, axis=1)
    assert v4.dtype == p_ifft
    # phase 5: unpad (and reduce, a no-op on one device) in p_unpad, output FP64
    v5 = v4[:, :Nt, :].astype(p_unpad).astype(np.float64)
    return v5[0] if squeeze else v5


def matvec_mixed(Fhat: np.ndarray, m: np.ndarray, Nt: int, prec: str) -> np.ndarray:
    """F m with the per-phase precisions named by ``prec`` (Section 3.2)."""
    return _mixed(Fhat, m, Nt, prec, adjoint=False)


def rmatvec_mixed(Fhat: np.ndarray, d: np.ndarray, Nt: int, prec: str) -> np.ndarray:
    """F* d with the per-phase precisions named by ``prec`` (Section 3.2).

    The letters name the phases in the order F* runs them: pad/FFT act on d,
    IFFT/unpad on the output m.
    """
    return _mixed(Fhat, d, Nt, prec, adjoint=True)


# ---------------------------------------------------------------------------
# Selected outputs, one at a time (full-size spot checks)
# ---------------------------------------------------------------------------

def matvec_entries(Fcol: np.ndarray, m: np.ndarray, idx) -> np.ndarray:
    """d_i[r] for each (i, r) in ``idx``, straight from the definition.

    d_i[r] = sum_{j<=i} sum_n F_{i-j}[r, n] m_j[n] (Section 2.3).  ``m`` is
    one right-hand side [Nt, Nm].
    """
    Fcol = np.asarray(Fcol)
    m = np.asarray(m, dtype=np.float64)
    out = np.empty(len(idx))
    for q, (i, r) in enumerate(idx):
        # rows F_{i-j}[r, :] for j = 0..i, i.e. lags k = i..0
        rows = np.asarray(Fcol[i::-1, r, :], dtype=np.float64)   # [i+1, Nm], row j holds F_{i-j}[r, :]
        out[q] = float(np.sum(rows * m[: i + 1]))
    return out


def rmatvec_entries(Fcol: np.ndarray, d: np.ndarray, idx) -> np.ndarray:
    """m*_j[n] for each (j, n) in ``idx``, straight from the definition.

    m*_j[n] = sum_{i>=j} sum_r F_{i-j}[r, n] d_i[r] (Section 2.3, F* = F^T).
    """
    Fcol = np.asarray(Fcol)
    d = np.asarray(d, dtype=np.float64)
    Nt = Fcol.shape[0]
    out = np.empty(len(idx))
    for q, (j, n) in enumerate(idx):
        cols = np.asarray(Fcol[: Nt - j, :, n], dtype=np.float64)  # [Nt-j, Nd], row k holds F_k[:, n]
        out[q] = float(np.sum(cols * d[j:]))
    return out


# ---------------------------------------------------------------------------
# Eq. (error), Section 3.2.1
# ---------------------------------------------------------------------------

EPS = {"s": 2.0 ** -24, "d": 2.0 ** -53}


def relative_error_bound(prec: str, Nt: int, n_inner: int, kappa: float, p: int = 1) -> float:
    """First-order relative error bound of Eq. (error) with every c_i = 1.

    kappa(F-hat) [ c1 e1 + (cF ed + c2 e2 + c4 e4) log2(Nt) + c3 e3 n + c5 e5 log2(p) ]
    with c1 = 0 when the pad phase is FP64 (a copy then adds no error) and
    n = n_m for F, n_d for F*.  ``prec`` is the 5-letter phase string.

    The paper counts unpad as an error-free memory operation, which holds in
    FP64; an FP32 unpad stores every output once in FP32, a relative rounding
    of e5 that the bound adds here (outside kappa, as it acts on the result
    itself).  This mirrors the c1 e1 term of the FP32 pad.
    """
    parse_precision(prec)
    e = [EPS[c] for c in prec]
    c1 = 0.0 if prec[0] == "d" else 1.0
    c5 = 0.0 if prec[4] == "d" else 1.0
    lg = np.log2(max(Nt, 2))
    bound = c1 * e[0] + (EPS["d"] + e[1] + e[3]) * lg + e[2] * n_inner
    if p > 1:
        bound += e[4] * np.log2(p)
    return float(kappa * bound + c5 * e[4])


def error_bound(prec: str, which: str, Nt: int, Nd: int, Nm: int, kappa: float, pr: int = 1, pc: int = 1) -> float:
    """Eq. (error) for one direction on a p_r x p_c process grid (Section 3.2.1).

    For F the block matvec's inner length is n_m = ceil(Nm / p_c) and the
    reduction of phase 5 runs over the p_c processes of a grid row; for F*
    the paper swaps in n_d = ceil(Nd / p_r) and p_r.  ``which`` is "F" or
    "F*".  Everything else is :func:`relative_error_bound`.
    """
    if which == "F":
        n, p = -(-Nm // pc), pc
    elif which == "F*":
        n, p = -(-Nd // pr), pr
    else:
        raise ValueError(f"which must be 'F' or 'F*', got {which!r}")
    return relative_error_bound(prec, Nt, n, kappa, p)


# ---------------------------------------------------------------------------
# Data-space Hessian, Section 2 (Gaussian prior and noise) and Remark 1
# ---------------------------------------------------------------------------

def hessian_entries(Fcol: np.ndarray, pairs, prior_var: float = 1.0, noise_var: float = 0.0) -> np.ndarray:
    """Entries of H_d = F G_prior F* + G_noise with isotropic covariances.

    G_prior = prior_var I and G_noise = noise_var I.  For data indices
    (t1, r1), (t2, r2) the block-Toeplitz structure gives
        H_d[(t1, r1), (t2, r2)] = prior_var sum_{j <= min(t1, t2)} sum_n F_{t1-j}[r1, n] F_{t2-j}[r2, n]
                                  + noise_var [t1 == t2 and r1 == r2],
    the inner product of rows (t1, r1) and (t2, r2) of the dense matrix.
    """
    Fcol = np.asarray(Fcol, dtype=np.float64)
    out = np.empty(len(pairs))
    for k, ((t1, r1), (t2, r2)) in enumerate(pairs):
        j = np.arange(min(t1, t2) + 1)
        acc = float(np.sum(Fcol[t1 - j, r1, :] * Fcol[t2 - j, r2, :]))
        out[k] = prior_var * acc + (noise_var if (t1, r1) == (t2, r2) else 0.0)
    return out
