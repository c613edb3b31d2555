"""Row-sharded rpCholesky-QR: A split into contiguous row blocks, one block per process.

Algorithm alg_2 (Section 4) with A partitioned by rows.  The row solves of both passes and the Gram
partials are row-local, so the processes exchange only two small objects:

  1. the s x n sample: every process writes the sampled rows it owns (zeros elsewhere) and the blocks
     are summed; each sample row has exactly one owner, so the sum is exact and every process
     factors the same sample into the same R_s;
  2. the n x n Gram partials A1_r^T A1_r: gathered and summed in rank order, so every process holds
     the same G and computes the same R1.

Q stays sharded like A; R is replicated.  The arithmetic of every step runs in the library's CUDA
kernels (``CudaSteps``); this module only orders the steps and the two exchanges.  A step backend
with the same methods can be substituted (the CPU tests drive the exchange logic with one).
"""
from __future__ import annotations

from typing import Protocol


class Comm(Protocol):
    world_size: int

    def allreduce_sum(self, t): ...

    def allgather(self, t) -> list: ...

    def allreduce_max_ints(self, v: list) -> list: ...


class TorchDistComm:
    """The two exchanges over torch.distributed (NCCL for CUDA tensors, gloo for CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world_size = dist.get_world_size(group)

    def allreduce_sum(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def allgather(self, t):
        parts = [t.new_empty(t.shape) for _ in range(self.world_size)]
        self.dist.all_gather(parts, t.contiguous(), group=self.group)
        return parts

    def allreduce_max_ints(self, v):
        import torch
        dev = "cpu" if self.dist.get_backend(self.group) == "gloo" else "cuda"
        t = torch.tensor([int(x) for x in v], dtype=torch.int64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return [int(x) for x in t.tolist()]


class SingleComm:
    """The exchanges of a one-process run: nothing to exchange."""
    world_size = 1

    def allreduce_sum(self, t):
        return t

    def allgather(self, t):
        return [t]

    def allreduce_max_ints(self, v):
        return [int(x) for x in v]


class CudaSteps:
    """The steps through the C ABI, on device tensors (an FP64 plan sized for the local block)."""

    def __init__(self, plan):
        from . import (rpcholqr_cholesky, rpcholqr_gather_owned_rows, rpcholqr_precondition_gram,
                       rpcholqr_sketch_r_from_sample, rpcholqr_solve_rows, rpcholqr_sum_partials,
                       rpcholqr_triu_mul)
        self.plan = plan
        self._gather = rpcholqr_gather_owned_rows
        self._sketch = rpcholqr_sketch_r_from_sample
        self._pre = rpcholqr_precondition_gram
        self._sum = rpcholqr_sum_partials
        self._chol = rpcholqr_cholesky
        self._solve = rpcholqr_solve_rows
        self._mul = rpcholqr_triu_mul

    def gather_owned(self, A_local, row_offset, m, s, seed):
        return self._gather(A_local, row_offset, m, s, seed)

    def sketch_r(self, As):
        return self._sketch(self.plan, As)

    def precondition_gram(self, A_local, Rs):
        return self._pre(self.plan, A_local, Rs)

    def sum_partials(self, parts):
        import torch
        return self._sum(torch.stack(parts).contiguous())

    def cholesky(self, G):
        return self._chol(self.plan, G)

    def solve_rows(self, A1, R1):
        return self._solve(self.plan, A1, R1, Y=A1)

    def triu_mul(self, R1, Rs):
        return self._mul(R1, Rs)

    @staticmethod
    def status(info) -> int:
        return int(info[0].item())


def factor_row_sharded(steps, comm: Comm, A_local, row_offset: int, m: int, s: int, seed: int):
    """(Q_local, R, status) of the row-sharded factorisation; every process calls it collectively.

    A_local holds the global rows row_offset .. row_offset + m_local - 1 of the m x n matrix A.
    status is the same on every process: the status of the first step, in step order, that failed on
    any process (0 = OK), so a NaN seen by one process is reported as NONFINITE everywhere rather than
    as the Cholesky breakdown it causes downstream."""
    # exchange 1: the sample
    As, info_g = steps.gather_owned(A_local, row_offset, m, s, seed)
    As = comm.allreduce_sum(As)
    Rs, info_s = steps.sketch_r(As)
    # local pass 1 and the Gram partial
    A1, G_local, info_p = steps.precondition_gram(A_local, Rs)
    # exchange 2: Gram partials, summed in rank order
    G = steps.sum_partials(comm.allgather(G_local))
    R1, info_c = steps.cholesky(G)
    Q_local, info_q = steps.solve_rows(A1, R1)
    R = steps.triu_mul(R1, Rs)
    per_step = comm.allreduce_max_ints([steps.status(i) for i in (info_g, info_s, info_p, info_c, info_q)])
    return Q_local, R, next((st for st in per_step if st), 0)


def split_rows(m: int, world_size: int, rank: int):
    """(row_offset, m_local) of rank's contiguous block in an even split (the first m % P blocks one
    row longer)."""
    base, extra = divmod(m, world_size)
    off = rank * base + min(rank, extra)
    return off, base + (1 if rank < extra else 0)
