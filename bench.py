#!/usr/bin/env python3
"""F / F* matvec throughput on the paper-shaped operator, one JSON line.

Workload: the paper-shaped single operator, Nt=1000, Nd=100, Nm=10000
(F-hat is 1001 x 100 x 10000 complex), block entries N(0,1) scaled by
exp(-k/200) over the lag k, one right-hand side m ~ N(0,1) for F and one
d ~ N(0,1) for F*.  A step is one F matvec and one F* matvec (every phase of
Section 2.4: pad, FFT, block matvec, IFFT, unpad), so a step is 2 matvecs.

value      matvecs/s over all ranks with inputs resident in HBM, device time
           from CUDA events on the launching stream; the headline precision
           is all-FP64-class (every phase FP64, the block matvec in the
           double-float FP32 hi/lo mode, relative L2 <= 1e-12 to the oracle).
e2e        the same metric through the public API with host (pinned) buffers,
           host<->device copies inside the timed region; consecutive steps
           alternate between two streams, so one step's copies (and FFTs)
           overlap the other's kernels.
roofline   the block-matvec kernels (about 90 % of a step): algorithmic bytes
           per launch (F-hat at its stored width + input + output vectors of
           one matvec) over their mean CUDA-event duration, against the
           measured HBM copy bandwidth.
variants   the plain FP64 path (native FP64 FMA), the paper's mixed-precision
           optimum, all-FP32, each with matvecs/s and its error.
paper_shape  the paper's own shape Nt=1000 Nd=100 Nm=5000 with the mantissa
           perturbation of Section 4.2.1: every phase configuration for F and
           F*, the Pareto front and the fastest under 1e-7 / 1e-5 / 1e-12.
rel_err    every error here is the relative L2 distance, over whole outputs,
           to the plain FP64 path (native FP64 FMA) run on the same inputs.
           That path's parity with the oracle, at these sizes and in this
           launch configuration, is checked by tests/test_fullsize.py; the
           GPU arm itself never runs the oracle.
multi_rhs  64 right-hand sides per call on the tensor cores (bf16 or FP16
           hi/lo), F and F*, with each kernel's time and DRAM bytes.
small      the plain FP64 Nt=64, Nd=8, Nm=32 workload: microseconds per matvec
           for the fused single launch and for the three-kernel path.
autograd   the differentiable adjoint Nt=500, Nd=200, Nm=5000 in FP32: loss +
           gradient (F forward, F* backward) per second, its HBM fraction and
           the gradient's error.
served     the four-operator served mix: capacity and p50/p99 latency.
cpu_baseline  the CPU oracle's FFT path on the whole operator (F-hat built
           and applied in blocks of rows), a few steps on all host cores.

--impl reference runs the CPU oracle itself (the only reference there is) on
the whole operator, timing exactly --steps steps after --warmup, and prints
the same line; only if those steps would take more than four minutes does it
fall back to a column sample (and says so in cpu_baseline.sample).
Multi-GPU (torchrun): every rank runs its own operator (no collective on the
data path), value = all matvecs / max-over-ranks time, scaling "weak".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NT, ND, NM = 1000, 100, 10000
DECAY = 200.0
METRIC = "F/F* matvec/s & HBM-roofline frac, Nt=1000 Nd=100 Nm=1e4; served p50/p99 ms"
UNIT = "matvec/s"
WORKLOAD = "paper-shaped single operator Nt=1000 Nd=100 Nm=10000, F and F* matvec, 1 RHS"
HEADLINE = ("ddddd", "f64x2f32", "f64x2f32")
# (phase string, block-matvec mode, FP64 FFT mode) for F and for F*
VARIANTS = {
    "fp64_native": (("ddddd", "native", "native"), ("ddddd", "native", "native")),
    "fp64_class_hilo": (("ddddd", "f64x2f32", "f64x2f32"), ("ddddd", "f64x2f32", "f64x2f32")),
    "fp64_class_gemv_native_fft": (("ddddd", "f64x2f32", "native"), ("ddddd", "f64x2f32", "native")),
    "paper_mp_optimum": (("dssdd", "native", "f64x2f32"), ("ddssd", "native", "f64x2f32")),
    "all_fp32": (("sssss", "native", "native"), ("sssss", "native", "native")),
}
# kernels of ours per headline matvec: the range check (largest magnitude of the
# input), the forward FFT, the block matvec and the inverse FFT (plus one
# cudaMemsetAsync of the range check's K words)
KERNELS_PER_MATVEC = 4
# mean DRAM bytes per launch of gemv_n_kernel / gemv_h_pipe_kernel <KindDF> at the paper
# shape (ncu dram__bytes read + write on Nm=2000, 3.239e9 and 3.214e9 B, scaled by 5 in Nm)
GEMV_DF_TRAFFIC = 16.13e9
# DRAM bytes (read + write) per K=64 bf16x2 call at the paper shape, per kernel, from
# ncu captures at Nm=2000 (profiles/fft_L2000_Nm2000_full.md, tc_gemm_k64_Nm2000_full.md)
# scaled by 5 in Nm where the traffic grows with Nm; the parts that do not (F*'s B planes
# of 100 data channels, the small FFTs over Nd channels) are taken at their algorithmic size
MULTI_RHS_DRAM = {
    "F": {"rfft_dif (B planes)": (0.5121 + 0.9915) * 5e9,
          "tc_gemm<0>": (1.602 + 1.1648) * 5e9 + 0.0499e9,   # A and B planes scale; D-hat out does not
          "irfft (Nd channels)": 64 * 1001 * 100 * 8 + 64 * 1000 * 100 * 4},
    "F*": {"rfft (Nd channels)": 64 * 1000 * 100 * 4 + 2 * 128 * 128 * 1001 * 2,
           "tc_gemm<1>": 1.602 * 5e9 + 0.066e9 + 0.9849 * 5e9,
           "irfft_dif": (1.0252 + 0.4812) * 5e9},
}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-multi", action="store_true")
    p.add_argument("--Nt", type=int, default=NT)
    p.add_argument("--Nd", type=int, default=ND)
    p.add_argument("--Nm", type=int, default=NM)
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# helpers shared with the multi-process tests
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (x itself when there is one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def algorithmic_bytes(Nt: int, Nd: int, Nm: int, fhat_entry_bytes: int, io_bytes: int = 8) -> int:
    """Bytes one matvec must move: F-hat at its stored width plus the input and
    output vectors (Nf = Nt + 1 frequencies of the paper's 2 Nt padding)."""
    Nf = Nt + 1
    return Nf * Nd * Nm * fhat_entry_bytes + Nt * Nm * io_bytes + Nt * Nd * io_bytes


def fhat_entry_bytes(prec: str, *modes: str) -> int:
    return 8 if prec[2] == "s" else 16


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[0]:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.REASONS, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def _blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return len(os.sched_getaffinity(0))


class OracleSample:
    """The oracle's FFT path on the first Nm_s columns of the operator (a bounded
    sample, for step counts too large to run the whole operator in minutes)."""

    def __init__(self, Fcol, m, d, Nm_s: int):
        import oracle
        self.oracle = oracle
        self.Nt = Fcol.shape[0]
        self.Nm_full = Fcol.shape[2]
        self.Nm_s = Nm_s
        self.Fh = oracle.spectrum(Fcol[:, :, :Nm_s])
        self.m = m[:, :Nm_s].copy()
        self.d = d.copy()
        self.scale = Nm_s / self.Nm_full

    def step(self):
        self.oracle.matvec_fft_spec(self.Fh, self.m, self.Nt)
        self.oracle.rmatvec_fft_spec(self.Fh, self.d, self.Nt)

    def time_steps(self, n: int) -> float:
        t0 = time.perf_counter()
        for _ in range(n):
            self.step()
        return time.perf_counter() - t0

    def describe(self) -> str:
        return (f"oracle FFT path (scipy.fft + numpy matmul, FP64) on columns 0..{self.Nm_s - 1} of the "
                f"Nm={self.Nm_full} operator (F-hat {self.Fh.nbytes / 1e9:.2f} GB), F + F* per step; "
                f"matvec/s scaled by {self.Nm_s}/{self.Nm_full} (work is linear in Nm)")


class OracleFull:
    """The oracle's FFT path on the whole operator.  F-hat (16 GB in FP64 at the
    paper shape) is built and applied in blocks of Nd rows, so no temporary
    exceeds one block: F gives each block's rows of d, F* sums the blocks'
    contributions F-hat_block^H d-hat_block (the inverse FFT is linear)."""

    def __init__(self, Fcol, m, d, rows_per_block: int = 25):
        import oracle
        self.oracle = oracle
        self.Nt, self.Nd, self.Nm = Fcol.shape
        self.blocks = [(r0, min(self.Nd, r0 + rows_per_block)) for r0 in range(0, self.Nd, rows_per_block)]
        t0 = time.perf_counter()
        self.Fh = [oracle.spectrum(Fcol[:, r0:r1, :]) for r0, r1 in self.blocks]
        self.setup_s = time.perf_counter() - t0
        self.m = m
        self.d = d
        self.scale = 1.0

    def step(self):
        import numpy as np
        dout = np.empty((self.Nt, self.Nd))
        for (r0, r1), Fh in zip(self.blocks, self.Fh):
            dout[:, r0:r1] = self.oracle.matvec_fft_spec(Fh, self.m, self.Nt)
        mout = np.zeros((self.Nt, self.Nm))
        for (r0, r1), Fh in zip(self.blocks, self.Fh):
            mout += self.oracle.rmatvec_fft_spec(Fh, self.d[:, r0:r1], self.Nt)
        return dout, mout

    def time_steps(self, n: int) -> float:
        t0 = time.perf_counter()
        for _ in range(n):
            self.step()
        return time.perf_counter() - t0

    def describe(self) -> str:
        gb = sum(f.nbytes for f in self.Fh) / 1e9
        return (f"oracle FFT path (scipy.fft + numpy matmul, FP64) on the whole Nt={self.Nt} Nd={self.Nd} "
                f"Nm={self.Nm} operator (F-hat {gb:.1f} GB in {len(self.blocks)} blocks of rows, built in "
                f"{self.setup_s:.1f} s, not timed), F + F* per step")


def _cpu_cores() -> int:
    return len(os.sched_getaffinity(0))


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(Fcol, m, d, steps: int = 3) -> dict:
    """The oracle's FFT path on the whole operator, a few steps, all host cores
    (FFT workers and BLAS threads)."""
    import scipy.fft
    cores = _cpu_cores()
    with scipy.fft.set_workers(cores):
        full = OracleFull(Fcol, m, d)
        full.step()                                  # warm-up
        t = full.time_steps(steps)
    rate = 2 * steps / t
    return {"value": rate, "unit": UNIT, "cores": cores, "blas_threads": _blas_threads(), "cpu": _cpu_model(),
            "kind": "oracle", "ms_per_step": 1e3 * t / steps,
            "sample": full.describe() + f"; {steps} steps in {t:.1f} s after one warm-up step"}


# the reference arm runs the whole operator when its steps fit this many seconds
REFERENCE_BUDGET_S = 240.0


def run_reference(args) -> None:
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import scipy.fft

    import synth
    Nt, Nd, Nm = args.Nt, args.Nd, args.Nm
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0, decay=DECAY)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=0)[0]
    d = synth.vectors(synth.TAG_D, Nt, Nd, seed=0)[0]
    cores = _cpu_cores()
    with scipy.fft.set_workers(cores):
        samp = OracleFull(Fcol, m, d)
        t1 = samp.time_steps(1)
        if (args.steps + args.warmup) * t1 > REFERENCE_BUDGET_S:
            # too many steps for the whole operator within minutes: a column sample
            Nm_s = max(8, int(Nm * REFERENCE_BUDGET_S / ((args.steps + args.warmup) * t1)))
            del samp
            samp = OracleSample(Fcol, m, d, Nm_s)
        samp.time_steps(args.warmup)
        t = samp.time_steps(args.steps)
    value = 2 * args.steps / t * samp.scale
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "Nt": Nt, "Nd": Nd, "Nm": Nm},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "blas_threads": _blas_threads(),
                         "cpu": _cpu_model(), "kind": "oracle", "sample": samp.describe()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def rel_diff(got, ref) -> float:
    """Relative L2 distance ||got - ref|| / ||ref|| of two device tensors (FP64)."""
    g, r = got.double(), ref.double()
    return float((g - r).norm() / r.norm())


def fp64_reference(op, x, which: str, stream):
    """The output of the plain FP64 path (every phase FP64, native FP64 FMA) for
    input x, the reference that the other precisions are measured against.
    Restores the operator's precision for `which` afterwards."""
    prev = op.get_precision(which)
    op.set_precision(which, "ddddd", "native", "native")
    call = op.matvec if which == "F" else op.rmatvec
    out = call(x.double(), stream=stream)
    op.set_precision(which, *prev)
    return out


def time_variant(torch, op, mt, dt, yt, xt, stream, pf, pa, steps: int) -> dict:
    op.set_precision("F", *pf)
    op.set_precision("F*", *pa)
    for _ in range(3):
        op.matvec(mt, out=yt, stream=stream)
        op.rmatvec(dt, out=xt, stream=stream)
    torch.cuda.synchronize()
    op.reset_timing()
    op.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        op.matvec(mt, out=yt, stream=stream)
        op.rmatvec(dt, out=xt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    op.set_timing(False)
    ms = e0.elapsed_time(e1)
    tf, nf = op.phase_times("F")
    ta, na = op.phase_times("F*")
    return {"ms_step": ms / steps, "matvec_s": 2 * steps / (ms * 1e-3),
            "gemv_ms_F": tf[1] / nf, "gemv_ms_Fstar": ta[1] / na,
            "phase_ms_F": [v / nf for v in tf], "phase_ms_Fstar": [v / na for v in ta]}


def bench_multi_rhs(torch, op, Fcol, dev, stream, peaks, which: str = "F", K: int = 64, steps: int = 10,
                    mode: str = "bf16x2") -> dict:
    """K right-hand sides through F (or F*) at once: FP32 phases, block matvec on
    the tensor cores with F-hat and the spectra split into bf16 (or FP16, scaled)
    hi + lo parts, the multi-RHS workload."""
    import numpy as np

    import synth
    Nt, Nd, Nm = Fcol.shape
    fwd = which == "F"
    n_in, n_out = (Nm, Nd) if fwd else (Nd, Nm)
    x = synth.vectors(synth.TAG_M if fwd else synth.TAG_D, Nt, n_in, k=K, seed=7, dtype=np.float32)
    xt = torch.from_numpy(x).to(dev)
    yt = torch.empty((K, Nt, n_out), dtype=torch.float32, device=dev)
    op.set_precision(which, "sssss", mode)
    call = op.matvec if fwd else op.rmatvec
    for _ in range(2):
        call(xt, out=yt, stream=stream)
    torch.cuda.synchronize()
    op.reset_timing()
    op.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call(xt, out=yt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    op.set_timing(False)
    ms = e0.elapsed_time(e1) / steps
    ph, n = op.phase_times(which)
    ph = [v / n for v in ph]
    # error on 8 of the K right-hand sides, whole outputs, against the plain FP64 path
    pick = torch.from_numpy(np.random.default_rng(5).choice(K, size=min(K, 8), replace=False)).to(dev)
    err = rel_diff(yt[pick], fp64_reference(op, xt[pick], which, stream))
    Nf, ldn, ldr = Nt + 1, (Nm + 7) // 8 * 8, (Nd + 7) // 8 * 8
    a_bytes = Nf * 4 * Nd * ldn * 2                    # bf16 hi/lo planes of F-hat
    # bf16 hi/lo [Re X | Im X] in, complex FP32 spectra out
    io_bytes = (Nf * 2 * 2 * K * ldn * 2 + K * Nf * Nd * 8) if fwd else (Nf * 2 * 2 * K * ldr * 2 + K * Nf * ldn * 8)
    tc_s = ph[1] * 1e-3
    if fwd:   # M = Nd rows per 128-row tile, contraction over ldn
        flops_exec = 6 * 2 * 128 * (2 * K) * ldn * Nf * ((Nd + 127) // 128)
    else:     # M = Nm rows, contraction over Nd in 64-wide steps
        flops_exec = 6 * 2 * 128 * (2 * K) * ((Nd + 63) // 64 * 64) * Nf * ((Nm + 127) // 128)
    hbm, _ = peaks
    bf16_peak = load_tensor_peak()
    tb = a_bytes + io_bytes
    desc = ("bf16 hi+lo" if mode == "bf16x2" else "FP16 hi+lo, power-of-two scale per frequency and per RHS")
    res = {"which": which, "K": K, "prec": f"sssss/{mode} (tcgen05, {desc}, FP32 accumulate)", "ms_call": ms,
            "matvec_s": K / (ms * 1e-3), "phase_ms": ph, "rel_err_8_rhs": err,
            "tc_kernel": {"hbm_bytes": tb, "achieved_GBs": tb / tc_s / 1e9,
                          "hbm_frac": tb / tc_s / 1e9 / hbm,
                          "tensor_TFLOPs_executed": flops_exec / tc_s / 1e12,
                          "tensor_frac": flops_exec / tc_s / 1e12 / bf16_peak,
                          "useful_TFLOPs": 8.0 * Nf * Nd * Nm * K / tc_s / 1e12},
            "algorithmic_bytes_per_call": int((Nt + 1) * Nd * Nm * 8 + K * Nt * Nm * 4 + K * Nt * Nd * 4)}
    if (Nt, Nd, Nm, K, mode) == (NT, ND, NM, 64, "bf16x2"):
        dram = MULTI_RHS_DRAM[which]
        res["dram_bytes_per_call"] = {"total": sum(dram.values()), "per_kernel": dram,
                                      "vs_algorithmic": sum(dram.values()) / res["algorithmic_bytes_per_call"],
                                      "source": "ncu dram__bytes read+write at Nm=2000, scaled to Nm=10000"}
    return res


def bench_small(torch, dev, calls: int = 2000) -> dict:
    """The plain FP64 workload Nt=64, Nd=8, Nm=32 (F-hat 266 KB, resident in L2):
    latency-bound, so it reports microseconds per call, issued directly and as
    a replayed CUDA graph of caller-scratch calls, for the fused single-launch
    path (one 16-CTA cluster per call, the default at this size) and for the
    three-kernel path, then the same in all-FP32 precision;
    a roofline fraction means nothing at this size."""
    import synth
    from paper_2508_10202_gb300 import Operator
    Nt, Nd, Nm = 64, 8, 32
    op = Operator(torch.from_numpy(synth.block_column(Nt, Nd, Nm, seed=0)).to(dev))
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, seed=0)[0]).to(dev)
    d = torch.from_numpy(synth.vectors(synth.TAG_D, Nt, Nd, seed=0)[0]).to(dev)
    y = torch.empty((Nt, Nd), dtype=torch.float64, device=dev)
    x = torch.empty((Nt, Nm), dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn) -> float:
        for _ in range(20):
            fn()
        torch.cuda.synchronize(dev)
        ev[0].record(s)
        for _ in range(calls // 2):
            fn()
        ev[1].record(s)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) * 1e3 / calls      # us per matvec

    def direct():
        op.matvec(m, out=y, stream=s)
        op.rmatvec(d, out=x, stream=s)

    def run() -> tuple[float, float]:
        us_direct = timed(direct)
        wf, wa = op.workspace_bytes("F", 1), op.workspace_bytes("F*", 1)
        ws = torch.empty(max(wf, wa) + 256, dtype=torch.uint8, device=dev)
        off = (-ws.data_ptr()) % 256
        wsf = ws[off:off + wf]
        wsa = ws[off:off + wa]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            op.apply_ws("F", m, y, wsf, stream=s)
            op.apply_ws("F*", d, x, wsa, stream=s)
        torch.cuda.synchronize(dev)
        with torch.cuda.graph(g, stream=s):
            op.apply_ws("F", m, y, wsf, stream=s)
            op.apply_ws("F*", d, x, wsa, stream=s)

        def graphed():
            with torch.cuda.stream(s):
                g.replay()
        return us_direct, timed(graphed)

    us_direct, us_graph = run()
    op.set_fusion(False)
    us_direct3, us_graph3 = run()
    # the same workload with every phase in FP32 (FP64 inputs and outputs)
    op.set_precision("F", "sssss")
    op.set_precision("F*", "sssss")
    op.set_fusion(True)
    f32_direct, f32_graph = run()
    op.set_fusion(False)
    f32_direct3, f32_graph3 = run()
    op.free()
    return {"workload": "plain FP64, Nt=64 Nd=8 Nm=32, F and F* alternating", "precision": "ddddd/native",
            "us_per_matvec_direct": us_direct, "us_per_matvec_graph": us_graph,
            "matvec_s_graph": 1e6 / us_graph, "path": "fused: one cluster launch per call",
            "three_kernel_path": {"us_per_matvec_direct": us_direct3, "us_per_matvec_graph": us_graph3},
            "fp32": {"precision": "sssss/native", "us_per_matvec_direct": f32_direct, "us_per_matvec_graph": f32_graph,
                     "three_kernel_path": {"us_per_matvec_direct": f32_direct3, "us_per_matvec_graph": f32_graph3}},
            "roofline": "not meaningful: launch- and latency-bound"}


def bench_hessian(torch, op, Fcol, stream, batch: int = 64, batches: int = 4) -> dict:
    """Data-space Hessian columns H_d e_i = F(F* e_i) + noise (Remark 1), batch unit
    vectors per F*/F pair on the tensor cores; the full matrix needs Nd*Nt columns."""
    import numpy as np

    from paper_2508_10202_gb300.hessian import hessian_columns
    Nt, Nd, Nm = Fcol.shape
    for w in ("F", "F*"):
        op.set_precision(w, "sssss", "bf16x2")
    rng = np.random.default_rng(11)
    idx = rng.choice(Nt * Nd, size=batch * (batches + 1), replace=False)
    with torch.cuda.stream(stream):
        hessian_columns(op, idx[:batch], noise_var=1e-4, batch=batch, dtype=torch.float32, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        cols = hessian_columns(op, idx[batch:], noise_var=1e-4, batch=batch, dtype=torch.float32, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) * 1e-3
    n = batch * batches
    # the first 8 timed columns again through the plain FP64 path
    for w in ("F", "F*"):
        op.set_precision(w, "ddddd", "native", "native")
    ref = hessian_columns(op, idx[batch:batch + 8], noise_var=1e-4, batch=8, stream=stream)
    return {"columns": n, "batch": batch, "seconds": s, "columns_per_s": n / s,
            "full_assembly_s_projected": Nt * Nd / (n / s),
            "prec": "sssss/bf16x2 both directions (tensor cores)",
            "rel_err_8_columns": rel_diff(cols[:8], ref)}


def bench_autograd(torch, dev, iters: int = 20) -> dict:
    """The differentiable-adjoint workload Nt=500, Nd=200, Nm=5000 in FP32: one
    loss + gradient of 1/2 ||F m - d||^2 is one F (forward) and one F* (backward,
    through autograd), each reading F-hat once (FP32, 4.0e9 B).  The gradient is
    compared with F*(F m - d) through the plain FP64 path."""
    import numpy as np

    import synth
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.autograd import toeplitz_matvec
    Nt, Nd, Nm = 500, 200, 5000
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0)
    op = Operator(Fcol)
    del Fcol
    m_true = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, seed=0)[0]).to(dev)
    op.set_precision("F", "ddddd", "native", "native")
    d_clean = op.matvec(m_true)
    noise = torch.from_numpy(synth.vectors(synth.TAG_NOISE, Nt, Nd, seed=0)[0]).to(dev)
    d = (d_clean + 0.01 * d_clean.norm() / (Nt * Nd) ** 0.5 * noise).float()
    m = torch.from_numpy(synth.vectors(synth.TAG_M, Nt, Nm, seed=1)[0]).to(dev).float().requires_grad_(True)
    for w in ("F", "F*"):
        op.set_precision(w, "sssss", "native", "native")

    def step():
        m.grad = None
        r = toeplitz_matvec(op, m) - d
        loss = 0.5 * (r * r).sum()
        loss.backward()
        return loss

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / iters
    g = m.grad.double()
    for w in ("F", "F*"):
        op.set_precision(w, "ddddd", "native", "native")
    md = m.detach().double()
    g64 = op.rmatvec(op.matvec(md) - d.double())
    op.free()
    fhat = (Nt + 1) * Nd * Nm * 8
    ab = 2 * (fhat + Nt * Nm * 4 + Nt * Nd * 4)
    peak, _ = load_peaks()
    return {"workload": "differentiable adjoint Nt=500 Nd=200 Nm=5000, FP32 (sssss), loss + gradient",
            "ms_per_loss_grad": ms, "loss_grads_per_s": 1e3 / ms,
            "algorithmic_bytes": ab, "hbm_frac": ab / (ms * 1e-3) / 1e9 / peak,
            "rel_err_grad": rel_diff(g, g64),
            "note": "the time includes the residual and loss arithmetic in PyTorch between the two matvecs"}


# the served mix: four resident operators (Nt, Nd, Nm), blocks N(0,1) in float32
SERVE_OPS = {"op128": (128, 16, 1000), "op256": (256, 64, 4000), "op500": (500, 100, 10000),
             "op1000": (1000, 200, 8000)}
SERVE_BUDGET = 150 * 10**9


def bench_serving(torch, dev, n_cap: int = 600, n_load: int = 2000, seed: int = 0) -> dict:
    """Poisson arrivals of F / F* requests (50/50, K ~ U{1..64}, operator uniform),
    admitted by a 150 GB HBM budget; capacity from a saturated run, then p50/p99
    at 0.5x and 0.9x of it."""
    import numpy as np

    import synth
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.serve import Request, Server, latency_stats
    t0 = time.perf_counter()
    ops = {}
    for i, (name, shp) in enumerate(SERVE_OPS.items()):
        col = synth.block_column(*shp, seed=100 + i, dtype=np.float32).astype(np.float64)
        ops[name] = Operator(col)
        del col
    setup_s = time.perf_counter() - t0
    srv = Server(ops, budget_bytes=SERVE_BUDGET, n_streams=4, keep_outputs=False)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    pools = {}
    for name, op in ops.items():
        pools[(name, "F")] = torch.randn((64, op.Nt, op.Nm), generator=gen, device=dev)
        pools[(name, "F*")] = torch.randn((64, op.Nt, op.Nd), generator=gen, device=dev)
    rng = np.random.default_rng(seed)
    names = list(ops)

    def requests(n):
        out = []
        for _ in range(n):
            name = names[rng.integers(len(names))]
            which = "F" if rng.random() < 0.5 else "F*"
            K = int(rng.integers(1, 65))
            out.append(Request(name, which, pools[(name, which)][:K]))
        return out

    for r in requests(48):              # warm-up: capture the graphs
        srv.submit(r)
    srv.run_until_idle()
    cap_reqs = requests(n_cap)          # capacity: everything arrives at once
    out = srv.run_schedule([(0.0, r) for r in cap_reqs])
    cap = latency_stats(out)
    mean_k = 32.5
    res = {"operators": {k: list(v) for k, v in SERVE_OPS.items()}, "budget_bytes": SERVE_BUDGET,
           "resident_bytes": srv.resident, "setup_s": setup_s, "precision": srv.precision,
           "capacity": cap}
    for frac in (0.5, 0.9):
        lam = frac * cap["matvec_s"] / mean_k          # requests per second
        reqs = requests(n_load)
        t = np.cumsum(rng.exponential(1.0 / lam, size=n_load))
        st = latency_stats(srv.run_schedule(list(zip(t, reqs))))
        st["offered_req_s"] = lam
        res[f"load_{frac}"] = st
    res["batches"] = srv.n_batches
    res["graph_batches"] = srv.n_graph_batches
    srv.close()
    for op in ops.values():
        op.free()
    return res


def bench_pareto(torch, op, mt, dt, yt, xt, stream) -> dict:
    """All 32 per-phase configurations (x the FP64 modes) for F and F*, timed and
    compared with the all-FP64 output; the Pareto front and the fastest
    configuration under the paper's 1e-7 tolerance and under 1e-5 / 1e-12."""
    from paper_2508_10202_gb300.pareto import best_under, pareto_front, sweep
    res = {}
    for which, x, out in (("F", mt, yt), ("F*", dt, xt)):
        op.set_precision(which, "ddddd", "native", "native")
        ref = (op.matvec(x, stream=stream) if which == "F" else op.rmatvec(x, stream=stream)).clone()
        pts = sweep(op, which, x, ref, reps=5, stream=stream)
        res[which] = {"n_configs": len(pts), "front": pareto_front(pts),
                      "best_1e-7": best_under(pts, 1e-7), "best_1e-5": best_under(pts, 1e-5),
                      "best_1e-12": best_under(pts, 1e-12)}
    return res


# the paper's own single-GPU shape (Section 4.1.2 and 4.2.1): Nt=1000, Nd=100, Nm=5000
PAPER_SHAPE = (1000, 100, 5000)


def bench_paper_shape(torch, dev, stream, reps: int = 20) -> dict:
    """The paper-comparable row: the Nt=1000, Nd=100, Nm=5000 operator with every
    block entry and input value given the mantissa perturbation of Section
    4.2.1 (fraction bits past the 23rd set to one), all phase configurations
    for F and F* timed (mean of `reps` calls) and measured against the plain
    FP64 output, as the paper's Pareto study does at its 1e-7 tolerance."""
    import synth
    from paper_2508_10202_gb300 import Operator
    from paper_2508_10202_gb300.pareto import best_under, pareto_front, sweep
    Nt, Nd, Nm = PAPER_SHAPE
    Fcol = synth.block_column(Nt, Nd, Nm, seed=0, decay=DECAY, perturb=True)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=0, perturb=True)[0]
    d = synth.vectors(synth.TAG_D, Nt, Nd, seed=0, perturb=True)[0]
    op = Operator(Fcol)
    del Fcol
    res = {"workload": "Nt=1000 Nd=100 Nm=5000, blocks N(0,1) x exp(-k/200), inputs N(0,1), all values with "
                       "the fraction bits past the 23rd set to one (Section 4.2.1)",
           "reps": reps, "reference": "plain FP64 GPU path (ddddd, native FP64 FMA)"}
    for which, x in (("F", torch.from_numpy(m).to(dev)), ("F*", torch.from_numpy(d).to(dev))):
        op.set_precision(which, "ddddd", "native", "native")
        ref = (op.matvec(x, stream=stream) if which == "F" else op.rmatvec(x, stream=stream)).clone()
        pts = sweep(op, which, x, ref, reps=reps, stream=stream)
        by = {(p["prec"], p["mode"], p["fft_mode"]): p for p in pts}
        base = by[("ddddd", "native", "native")]
        fp64c = by[("ddddd", "f64x2f32", "f64x2f32")]
        opt = "dssdd" if which == "F" else "ddssd"
        best7 = best_under(pts, 1e-7)
        res[which] = {
            "n_configs": len(pts), "front": pareto_front(pts),
            "fp64_native": base, "fp64_class": fp64c,
            "paper_optimum": {k: by.get((opt, "native", k)) for k in ("native", "f64x2f32")},
            "best_1e-7": best7, "best_1e-5": best_under(pts, 1e-5), "best_1e-12": best_under(pts, 1e-12),
            "speedup_best_1e-7_vs_fp64_native": base["ms"] / best7["ms"] if best7 else None,
            "speedup_best_1e-7_vs_fp64_class": fp64c["ms"] / best7["ms"] if best7 else None,
        }
    op.free()
    return res


def load_tensor_peak() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def main(args) -> None:
    import numpy as np
    import torch

    import synth
    from paper_2508_10202_gb300 import Operator

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    Nt, Nd, Nm = args.Nt, args.Nd, args.Nm
    seed = rank

    t0 = time.perf_counter()
    Fcol = synth.block_column(Nt, Nd, Nm, seed=seed, decay=DECAY)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=seed)[0]
    d = synth.vectors(synth.TAG_D, Nt, Nd, seed=seed)[0]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    op = Operator(Fcol)                      # host block column: staged setup FFT in FP64
    t_setup = time.perf_counter() - t0

    stream = torch.cuda.current_stream(dev)
    mt = torch.from_numpy(m).to(dev)
    dt = torch.from_numpy(d).to(dev)
    yt = torch.empty((Nt, Nd), dtype=torch.float64, device=dev)
    xt = torch.empty((Nt, Nm), dtype=torch.float64, device=dev)

    # --- headline: timed region, max over ranks --------------------------------
    op.set_precision("F", *HEADLINE)
    op.set_precision("F*", *HEADLINE)
    for _ in range(args.warmup):
        op.matvec(mt, out=yt, stream=stream)
        op.rmatvec(dt, out=xt, stream=stream)
    op.set_timing(True)
    op.reset_timing()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        op.matvec(mt, out=yt, stream=stream)
        op.rmatvec(dt, out=xt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    units = sum_over_ranks(2.0 * args.steps, world, dev)
    value = units / (ms_max * 1e-3)
    tf, nf = op.phase_times("F")
    ta, na = op.phase_times("F*")
    op.set_timing(False)
    y = yt.cpu().numpy()
    x = xt.cpu().numpy()
    y64 = fp64_reference(op, mt, "F", stream)
    x64 = fp64_reference(op, dt, "F*", stream)
    err_f, err_a = rel_diff(yt, y64), rel_diff(xt, x64)

    # --- roofline of the block-matvec kernels ----------------------------------
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(Nt, Nd, Nm, fhat_entry_bytes(*HEADLINE))
    gemv_ms = (tf[1] + ta[1]) / (nf + na)
    achieved = ab / (gemv_ms * 1e-3) / 1e9
    # DRAM bytes per launch of the same two kernels from ncu --set full at Nm=2000,
    # scaled x5 to the full operator (profiles/gemv_df_paper_shape_Nm2000_full.md)
    traffic = GEMV_DF_TRAFFIC if (Nt, Nd, Nm) == (NT, ND, NM) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "gemv_n_kernel<KindDF> (F) / gemv_h_pipe_kernel<KindDF> (F*)",
                "bytes_per_launch": ab, "gemv_ms_F": tf[1] / nf, "gemv_ms_Fstar": ta[1] / na,
                "frac_F": ab / (tf[1] / nf * 1e-3) / 1e9 / peak, "frac_Fstar": ab / (ta[1] / na * 1e-3) / 1e9 / peak,
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "phase_ms_F": [v / nf for v in tf], "phase_ms_Fstar": [v / na for v in ta]}

    # --- end to end through the public API with host buffers -------------------
    mh = torch.from_numpy(m).pin_memory()
    dh = torch.from_numpy(d).pin_memory()
    yh = torch.empty((Nt, Nd), dtype=torch.float64).pin_memory()
    xh = torch.empty((Nt, Nm), dtype=torch.float64).pin_memory()
    for _ in range(3):
        op.matvec(mh, out=yh)
        op.rmatvec(dh, out=xh)
    # all host buffers pinned, so the calls are stream ordered: consecutive steps
    # alternate between two streams, each with its own pinned inputs and outputs,
    # and one step's host copies overlap the other's kernels
    e2e_steps = max(10, min(args.steps, 100))
    e2e_streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    bufs = [(mh, dh, yh, xh), (mh.clone().pin_memory(), dh.clone().pin_memory(),
                               torch.empty_like(yh).pin_memory(), torch.empty_like(xh).pin_memory())]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        st = e2e_streams[i % 2]
        mi, di, yi, xi = bufs[i % 2]
        op.matvec(mi, out=yi, stream=st)
        op.rmatvec(di, out=xi, stream=st)
    torch.cuda.synchronize(dev)
    t_e2e = time.perf_counter() - t0
    assert np.allclose(bufs[(e2e_steps - 1) % 2][2].numpy(), y, rtol=0, atol=1e-9 * np.abs(y).max())
    t_e2e = max_over_ranks(t_e2e, world, dev)
    e2e = {"value": sum_over_ranks(2.0 * e2e_steps, world, dev) / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(m.nbytes + d.nbytes), "d2h_bytes_per_step": int(y.nbytes + x.nbytes),
           "steps": e2e_steps}

    # --- variants (rank 0 only) --------------------------------------------------
    variants = {}
    if rank == 0 and not args.no_variants:
        for name, (pf, pa) in VARIANTS.items():
            r = time_variant(torch, op, mt, dt, yt, xt, stream, pf, pa, steps=max(20, args.steps // 5))
            ef, ea = rel_diff(yt, y64), rel_diff(xt, x64)
            abv = algorithmic_bytes(Nt, Nd, Nm, fhat_entry_bytes(*pf))
            r.update({"prec_F": "/".join(pf), "prec_Fstar": "/".join(pa), "rel_err_F": ef, "rel_err_Fstar": ea,
                      "gemv_frac_F": abv / (r["gemv_ms_F"] * 1e-3) / 1e9 / peak,
                      "gemv_frac_Fstar": abv / (r["gemv_ms_Fstar"] * 1e-3) / 1e9 / peak})
            variants[name] = r

    pareto = None
    if rank == 0 and not args.no_variants:
        pareto = bench_pareto(torch, op, mt, dt, yt, xt, stream)

    paper_shape = None
    if rank == 0 and not args.no_variants and (Nt, Nd, Nm) == (NT, ND, NM):
        paper_shape = bench_paper_shape(torch, dev, stream)

    multi = None
    if rank == 0 and not args.no_multi:
        multi = {w: bench_multi_rhs(torch, op, Fcol, dev, stream, (peak, peak_kind), which=w) for w in ("F", "F*")}
        for w in ("F", "F*"):
            multi[w + " f16x2"] = bench_multi_rhs(torch, op, Fcol, dev, stream, (peak, peak_kind), which=w, mode="f16x2")

    hess = None
    if rank == 0 and not args.no_multi:
        hess = bench_hessian(torch, op, Fcol, stream)

    small = None
    autograd = None
    if rank == 0 and not args.no_variants:
        small = bench_small(torch, dev)
        autograd = bench_autograd(torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(Fcol, m, d)

    served = None
    if rank == 0 and not args.no_serve:
        op.free()                       # make room for the served operators
        del mt, dt, yt, xt
        torch.cuda.empty_cache()
        served = bench_serving(torch, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2 (FP64-class double-float on the FP32 pipe)",
            "data": "synthetic (seeded N(0,1) blocks x exp(-k/200), N(0,1) vectors)",
            "config": {"workload": WORKLOAD, "Nt": Nt, "Nd": Nd, "Nm": Nm, "rhs": 1,
                       "precision": "ddddd, block matvec and FFTs in f64x2f32", "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2: F-hat is 16 GB per matvec, read once"},
            "gpu_launches": KERNELS_PER_MATVEC * 2 * args.steps,
            "rel_err": {"F": err_f, "Fstar": err_a,
                        "how": "relative L2 over the whole outputs against the plain FP64 path (native FP64 FMA) "
                               "on the same inputs; that path's parity with the oracle is tests/test_fullsize.py"},
            "roofline": roofline, "e2e": e2e, "clocks": clk, "cpu_baseline": cpu, "variants": variants,
            "multi_rhs": multi, "hessian": hess, "small": small, "autograd": autograd, "pareto": pareto,
            "paper_shape": paper_shape,
            "served": served,
            "served_p50_ms": served["load_0.9"]["p50_ms"] if served else None,
            "served_p99_ms": served["load_0.9"]["p99_ms"] if served else None,
            "setup_s": t_setup, "gen_s": t_gen,
        }
        print(json.dumps(line), flush=True)
    if served is None:
        op.free()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    else:
        main(a)
