"""Row-sharded factorisation on CPU ranks (gloo, world sizes 2 and 3): the exchange logic of
paper_2406_11751_gb300.sharded driven by an oracle-backed step backend.

Pins: the summed sample equals the oracle's single-process sample bit for bit (every sample row has
one owner, so the sum is exact), hence R_s is identical; the A_1 rows are identical (row solves are
row-local); the Gram matrix, summed from per-rank partials in rank order, agrees to rounding
(1e-14 relative), and Q, R to 1e-12; every rank reports the same status, including a NaN that only
one rank owns.
"""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import inputs

pytestmark = pytest.mark.timeout(300) if hasattr(pytest.mark, "timeout") else []


class OracleSteps:
    """The steps of the sharded driver computed by the FP64 oracle on CPU tensors."""

    def __init__(self, oracle):
        self.o = oracle

    def gather_owned(self, A_local, row_offset, m, s, seed):
        A = A_local.numpy()
        idx = self.o.sample_indices(seed, m, s) - row_offset
        own = (idx >= 0) & (idx < A.shape[0])
        As = np.zeros((s, A.shape[1]))
        if own.any():
            As[own] = np.sqrt(m / s) * A[idx[own]]       # the scale of Remark r_exp, global m and s
        bad = not np.all(np.isfinite(A[idx[own]]))
        return torch.from_numpy(As), torch.tensor([2 if bad else 0, -1])

    def sketch_r(self, As):
        Rs, st = self.o.householder_r(As.numpy())
        return torch.from_numpy(Rs), torch.tensor([st, -1])

    def precondition_gram(self, A_local, Rs):
        A1 = self.o.trsm_rows(A_local.numpy(), Rs.numpy())
        bad = not np.all(np.isfinite(A_local.numpy()))
        return torch.from_numpy(A1), torch.from_numpy(self.o.gram(A1)), torch.tensor([2 if bad else 0, -1])

    def sum_partials(self, parts):
        G = parts[0].clone()
        for p in parts[1:]:
            G += p
        return G

    def cholesky(self, G):
        R1, st, piv = self.o.cholesky_upper(G.numpy())
        return torch.from_numpy(R1), torch.tensor([st, piv])

    def solve_rows(self, A1, R1):
        return torch.from_numpy(self.o.trsm_rows(A1.numpy(), R1.numpy())), torch.tensor([0, -1])

    def triu_mul(self, R1, Rs):
        return torch.from_numpy(self.o.triu_mul(R1.numpy(), Rs.numpy()))

    @staticmethod
    def status(info):
        return int(info[0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, A, s, seed, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2406_11751_gb300.sharded import TorchDistComm, factor_row_sharded, split_rows
        m = A.shape[0]
        off, ml = split_rows(m, world, rank)
        steps = OracleSteps(oracle)
        comm = TorchDistComm()
        As, _ = steps.gather_owned(torch.from_numpy(A[off:off + ml]), off, m, s, seed)
        As_sum = comm.allreduce_sum(As.clone())
        Q, R, st = factor_row_sharded(steps, comm, torch.from_numpy(np.ascontiguousarray(A[off:off + ml])),
                                      off, m, s, seed)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), Q=Q.numpy(), R=R.numpy(), st=st, off=off,
                 As=As_sum.numpy())
    finally:
        dist.destroy_process_group()


def _run(world, A, s, seed):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), A, s, seed, d), nprocs=world, join=True,
                           start_method="spawn")
        return [dict(np.load(os.path.join(d, f"r{r}.npz"))) for r in range(world)]


@pytest.mark.parametrize("world,m,n,kappa", [(2, 3001, 20, 1e8), (3, 2500, 16, 1e12), (2, 401, 40, 1e4)])
def test_row_sharded_matches_single_process(oracle_mod, world, m, n, kappa):
    A = inputs.usv(m, n, kappa, 40 + world)
    s, seed = 3 * n, 9
    outs = _run(world, A, s, seed)
    o = oracle_mod.rpcholqr(A, s, seed, intermediates=True)
    As_ref = oracle_mod.gather_scale(A, oracle_mod.sample_indices(seed, m, s))
    Q = np.concatenate([r["Q"] for r in outs])
    for r in outs:
        assert int(r["st"]) == 0
        assert np.array_equal(r["As"], As_ref)              # exchange 1 is exact
        assert np.array_equal(r["R"], outs[0]["R"])          # R replicated bit for bit
    assert np.linalg.norm(outs[0]["R"] - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
    if kappa <= 1e8:
        floor = np.linalg.norm(o["Q"] - oracle_mod.rpcholqr(A, s, seed, variant=1)["Q"], 2)
        assert np.linalg.norm(Q - o["Q"], 2) <= max(1e-10, 10 * floor)
    assert oracle_mod.orth_error(Q) <= 10 * oracle_mod.orth_error(o["Q"])


def test_row_sharded_status_agrees_across_ranks(oracle_mod):
    m, n, s, seed = 2000, 12, 36, 4
    A = inputs.usv(m, n, 10.0, 3)
    idx = set(oracle_mod.sample_indices(seed, m, s).tolist())
    # a NaN in a row outside the sample, in the second rank's block: only rank 1 sees it in pass 1
    A[next(i for i in range(1500, m) if i not in idx), 5] = np.nan
    outs = _run(2, A, s, seed)
    assert [int(r["st"]) for r in outs] == [2, 2]


def test_split_rows_covers_every_row():
    from paper_2406_11751_gb300.sharded import split_rows
    for m in (1, 7, 100, 1001):
        for p in (1, 2, 3, 8):
            if m < p:
                continue
            blocks = [split_rows(m, p, r) for r in range(p)]
            assert blocks[0][0] == 0
            for (o1, l1), (o2, _) in zip(blocks, blocks[1:]):
                assert o1 + l1 == o2
            assert sum(l for _, l in blocks) == m
            assert max(l for _, l in blocks) - min(l for _, l in blocks) <= 1


def test_single_process_comm_matches_a_one_rank_group(oracle_mod):
    # bench.py --sharded at N = 1 runs the driver without a process group: SingleComm must give what a
    # one-rank group gives (the identity exchanges), so the result equals the whole-matrix oracle run
    from paper_2406_11751_gb300.sharded import SingleComm, factor_row_sharded
    A = inputs.usv(1500, 12, 1e6, 3)
    comm = SingleComm()
    t = torch.ones(3)
    assert comm.allreduce_sum(t) is t and comm.allgather(t) == [t] and comm.allreduce_max_ints([0, 4]) == [0, 4]
    Q, R, st = factor_row_sharded(OracleSteps(oracle_mod), comm, torch.from_numpy(A), 0, 1500, 36, 5)
    o = oracle_mod.rpcholqr(A, 36, 5)
    assert st == 0 and np.array_equal(R.numpy(), o["R"]) and np.array_equal(Q.numpy(), o["Q"])
