"""Distribution of F over a p_r x p_c process grid (Section 2.4).

The paper partitions the operator's blocks by sensor rows (Nd, over p_r
process rows) and parameter columns (Nm, over p_c process columns).  Rank
(i, j) holds the block F^(i,j) = F[:, rows_i, cols_j] of the first block
column and the column slice m^(j) of the parameter vector.  Then
    F m:   d^(i) = sum_j F^(i,j) m^(j)        (phase 5: reduce over the p_c
                                               ranks of process row i)
    F* d:  m^(j) = sum_i F^(i,j)* d^(i)       (phase 1 broadcasts d^(i) along
                                               the process row; phase 5 reduces
                                               over the p_r ranks of column j)
With p_r = 1 (the paper's choice up to about 512 GPUs) F* needs only the
broadcast of d.  The local products run on each rank's own operator (a GPU
``Operator``, or any object with ``matvec``/``rmatvec``); the exchanges use
``torch.distributed`` collectives.

Every GPU machine of this project has one GPU, so benchmarks run one independent
operator per rank; this module and its multi-process CPU tests (gloo) keep
the partition math and the collectives honest.
"""
from __future__ import annotations

import math

__all__ = ["grid_shape", "shard_bounds", "local_block", "ShardedOperator"]


def grid_shape(p: int) -> tuple[int, int]:
    """Process grid (p_r, p_c) for p processes.

    Section 4.2.2: one process row up to 512 GPUs, eight rows at 1024 and 2048
    GPUs, sixteen at 4096 (the communication-aware choice reported for Frontier).
    In between, rows double with p past 512.
    """
    if p < 1:
        raise ValueError("p must be >= 1")
    if p <= 512:
        return 1, p
    pr = 8 if p <= 2048 else 16
    while p % pr:
        pr //= 2
    return pr, p // pr


def shard_bounds(n: int, parts: int, idx: int) -> tuple[int, int]:
    """Half-open range of the idx-th of `parts` contiguous blocks of n items.

    Blocks hold ceil(n / parts) items except at the end (the n_m = ceil(Nm / p_c)
    of Section 3.2.1); trailing blocks may be empty when parts does not divide n.
    """
    if not 0 <= idx < parts:
        raise ValueError("idx out of range")
    size = math.ceil(n / parts)
    lo = min(n, idx * size)
    return lo, min(n, lo + size)


def local_block(F_col, rank: int, pr: int, pc: int):
    """The block column slice F_col[:, rows_i, cols_j] owned by `rank` (row-major grid)."""
    i, j = divmod(rank, pc)
    Nd, Nm = F_col.shape[1], F_col.shape[2]
    r0, r1 = shard_bounds(Nd, pr, i)
    c0, c1 = shard_bounds(Nm, pc, j)
    return F_col[:, r0:r1, c0:c1]


class ShardedOperator:
    """F and F* on a p_r x p_c grid of ranks, each holding one operator block.

    ``local`` computes the rank's block products; ``row_group`` holds the p_c
    ranks of this rank's process row, ``col_group`` the p_r ranks of its
    process column (``None`` means the default group).  Vectors are
    torch tensors; m is sliced by columns, d by rows.
    """

    def __init__(self, local, rank: int, pr: int, pc: int, row_group=None, col_group=None, row_src: int | None = None):
        self.local = local
        self.rank = rank
        self.pr, self.pc = pr, pc
        self.i, self.j = divmod(rank, pc)
        self.row_group, self.col_group = row_group, col_group
        # global rank that owns d^(i) before the phase-1 broadcast along process row i
        self.row_src = self.i * pc if row_src is None else row_src

    def matvec(self, m_local):
        """d^(i) = sum_j F^(i,j) m^(j): local product, then sum over the process row."""
        import torch.distributed as dist
        d = self.local.matvec(m_local)
        if self.pc > 1:
            dist.all_reduce(d, op=dist.ReduceOp.SUM, group=self.row_group)
        return d

    def rmatvec(self, d_local):
        """m^(j) = sum_i F^(i,j)* d^(i): broadcast d^(i) along the row, local product,
        then sum over the process column."""
        import torch.distributed as dist
        if self.pc > 1:
            dist.broadcast(d_local, src=self.row_src, group=self.row_group)
        m = self.local.rmatvec(d_local)
        if self.pr > 1:
            dist.all_reduce(m, op=dist.ReduceOp.SUM, group=self.col_group)
        return m
