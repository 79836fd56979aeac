"""Host-side pieces of bench.py (no GPU): the CPU baseline's blocked oracle run
and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_blocked_oracle_equals_direct():
    import bench
    Nt, Nd, Nm = 16, 7, 9
    Fcol = synth.block_column(Nt, Nd, Nm, seed=4, decay=200.0)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=4)[0]
    d = synth.vectors(synth.TAG_D, Nt, Nd, seed=4)[0]
    full = bench.OracleFull(Fcol, m, d, rows_per_block=3)
    assert len(full.blocks) == 3 and full.blocks[-1] == (6, 7)
    y, x = full.step()
    assert oracle.rel_l2(y, oracle.matvec_direct(Fcol, m)) <= 1e-13
    assert oracle.rel_l2(x, oracle.rmatvec_direct(Fcol, d)) <= 1e-13


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--Nt", "16",
                        "--Nd", "5", "--Nm", "12", "--steps", "3", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "whole" in line["cpu_baseline"]["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the timed steps are the whole operator: value and ms_per_step agree
    assert abs(line["value"] - 2e3 / line["ms_per_step"]) <= 1e-6 * line["value"]
    assert np.isfinite(line["value"])


def test_reference_arm_under_two_ranks():
    # launched as the multi-GPU bench is (torch.distributed.run, 2 ranks): rank
    # 0 alone times the oracle and prints the one line, the other exits 0
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--Nt", "16", "--Nd", "5", "--Nm", "12",
                        "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 2
    assert line["value"] > 0


def _rank_reduce_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = (bench.max_over_ranks(1.5 + rank, world), bench.sum_over_ranks(1.5 + rank, world))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_reductions_gloo():
    # the GPU arm's time is the maximum over ranks and its units the sum, on
    # every rank (gloo on CPU here; NCCL on the GPU machine)
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    world = 3
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_reduce_worker, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got == {r: (3.5, 7.5) for r in range(world)}
    import bench
    assert bench.max_over_ranks(2.0, 1) == 2.0 and bench.sum_over_ranks(2.0, 1) == 2.0
