"""Pareto-front selection of per-phase precisions (Sections 3.2 and 4.2.1).

Each of the five phases (pad, FFT, block matvec, IFFT, unpad) runs in FP32 or
FP64: 32 configurations; on GB300 every FP64 phase can also use the
double-float FP32-pipe mode, which the sweep includes.  Every configuration
is timed (CUDA events, mean of ``reps`` calls) and its relative L2 error is
measured against a reference output (the paper uses the all-FP64 output).
The Pareto front keeps the configurations no other one beats in both time and
error; ``best_under`` picks the fastest with error below a tolerance.
"""
from __future__ import annotations

import itertools

import torch

__all__ = ["CONFIGS", "sweep", "pareto_front", "best_under"]

CONFIGS = ["".join(p) for p in itertools.product("ds", repeat=5)]


def _modes(prec: str):
    """(block-matvec mode, FFT mode) pairs: native FP64 everywhere, and the
    FP64-class mode wherever an FP64 phase can use it."""
    f64_gemv = prec[2] == "d"
    f64_fft = prec[1] == "d" or prec[3] == "d"
    if not (f64_gemv or f64_fft):
        return [("native", "native")]
    return [("native", "native"), ("f64x2f32" if f64_gemv else "native", "f64x2f32" if f64_fft else "native")]


def sweep(op, which: str, x: torch.Tensor, ref: torch.Tensor, reps: int = 10, configs=None, stream=None):
    """Time and error of every configuration for F (which="F") or F* on input x."""
    s = torch.cuda.current_stream() if stream is None else stream
    fn = op.matvec if which == "F" else op.rmatvec
    out = torch.empty_like(ref, dtype=x.dtype)
    refn = ref.double()
    denom = float(refn.norm())
    results = []
    for prec in (configs or CONFIGS):
        for gm, fm in _modes(prec):
            op.set_precision(which, prec, gm, fm)
            fn(x, out=out, stream=s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn(x, out=out, stream=s)
            e1.record(s)
            e1.synchronize()
            err = float((out.double() - refn).norm()) / denom
            results.append({"prec": prec, "mode": gm, "fft_mode": fm, "ms": e0.elapsed_time(e1) / reps, "rel_err": err})
    return results


def pareto_front(points: list[dict]) -> list[dict]:
    """Points not dominated in (ms, rel_err), sorted by time."""
    pts = sorted(points, key=lambda p: (p["ms"], p["rel_err"]))
    front, best_err = [], float("inf")
    for p in pts:
        if p["rel_err"] < best_err:
            front.append(p)
            best_err = p["rel_err"]
    return front


def best_under(points: list[dict], tol: float) -> dict | None:
    """The fastest configuration whose error is at most tol."""
    ok = [p for p in points if p["rel_err"] <= tol]
    return min(ok, key=lambda p: p["ms"]) if ok else None
