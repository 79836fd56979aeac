"""The p_r x p_c partition of Section 2.4 with real collectives (gloo ranks on CPU).

Each rank owns one block F^(i,j) of the first block column; its local
products come from the CPU oracle through a small adapter (test side), so
these tests exercise the partition math and the phase-1 broadcast / phase-5
reductions of ShardedOperator without a GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2508_10202_gb300.distributed import ShardedOperator, grid_shape, local_block, shard_bounds

NT, ND, NM = 12, 7, 23


class OracleBlock:
    """Local products of one operator block by the CPU oracle (test adapter)."""

    def __init__(self, F):
        self.F = F

    def matvec(self, m):
        return torch.from_numpy(oracle.matvec_direct(self.F, m.numpy()))

    def rmatvec(self, d):
        return torch.from_numpy(oracle.rmatvec_direct(self.F, d.numpy()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, pr, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pc = world // pr
    rows = [dist.new_group([i * pc + j for j in range(pc)]) for i in range(pr)]
    cols = [dist.new_group([i * pc + j for i in range(pr)]) for j in range(pc)]
    i, j = divmod(rank, pc)
    F = synth.block_column(NT, ND, NM, seed=3)
    m = synth.vectors(synth.TAG_M, NT, NM, seed=3)[0]
    d = synth.vectors(synth.TAG_D, NT, ND, seed=3)[0]
    r0, r1 = shard_bounds(ND, pr, i)
    c0, c1 = shard_bounds(NM, pc, j)
    sop = ShardedOperator(OracleBlock(local_block(F, rank, pr, pc)), rank, pr, pc, rows[i], cols[j])
    d_i = sop.matvec(torch.from_numpy(m[:, c0:c1].copy()))
    assert oracle.rel_l2(d_i.numpy(), oracle.matvec_direct(F, m)[:, r0:r1]) <= 1e-13
    # only the row's source rank holds d^(i) before the broadcast
    d_in = torch.from_numpy(d[:, r0:r1].copy()) if j == 0 else torch.zeros((NT, r1 - r0), dtype=torch.float64)
    m_j = sop.rmatvec(d_in)
    assert oracle.rel_l2(m_j.numpy(), oracle.rmatvec_direct(F, d)[:, c0:c1]) <= 1e-13
    dist.barrier()
    dist.destroy_process_group()


# 1 x 2: the row reduction; 2 x 1: the column reduction with one-rank row
# groups; 2 x 2: the broadcast and both reductions
@pytest.mark.parametrize("world,pr", [(2, 1), (2, 2), (4, 2)])
def test_sharded_operator_gloo(world, pr):
    mp.spawn(_worker, args=(world, pr, _free_port()), nprocs=world, join=True)


def test_grid_and_bounds():
    assert grid_shape(1) == (1, 1) and grid_shape(512) == (1, 512)
    assert grid_shape(1024) == (8, 128) and grid_shape(2048) == (8, 256) and grid_shape(4096) == (16, 256)
    for n in (1, 7, 100, 10000):
        for parts in (1, 2, 3, 8):
            spans = [shard_bounds(n, parts, k) for k in range(parts)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(hi - lo for lo, hi in spans) == -(-n // parts)
    with pytest.raises(ValueError):
        shard_bounds(5, 2, 2)
