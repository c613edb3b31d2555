"""GPU tests of the batched entry points: many independent matrices of uneven m and n.

Each matrix of a batch runs the same kernels as a single rpcholqr_factor call with the same plan
limits, so the batched results -- dealt round-robin over concurrent slots, or captured into a CUDA
graph and replayed -- must be bit-identical to the single calls, and match the oracle like them.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

SHAPES = [(4096, 8), (30011, 128), (5000, 16), (70001, 64), (8192, 32), (12000, 100), (4500, 8),
          (20000, 50), (4096, 128), (9000, 1), (100000, 16), (6000, 77)]


def _make_batch():
    As, ss, seeds = [], [], []
    for i, (m, n) in enumerate(SHAPES):
        As.append(torch.from_numpy(inputs.usv(m, n, 10.0 ** (i % 14), 40 + i)).to(DEV))
        ss.append(3 * n)
        seeds.append(1000 + i)
    return As, ss, seeds


@pytest.mark.parametrize("mode_name", ["FP64", "SPLIT64"])
def test_batched_equals_single_calls(lib, mode_name):
    mode = getattr(lib, mode_name)
    As, ss, seeds = _make_batch()
    batch = lib.rpcholqr_batch_create(0, 1 << 17, 128, 384, slots=4, mode=mode)
    plan = lib.rpcholqr_plan_create(0, 1 << 17, 128, 384, mode=mode)
    try:
        Qs, Rs, info = lib.rpcholqr_batch_factor(batch, As, ss, seeds)
        torch.cuda.synchronize()
        st = info.cpu().view(-1, 2).tolist()
        assert all(x == [0, -1] for x in st), st
        for A, s, seed, Q, R in zip(As, ss, seeds, Qs, Rs):
            Q1, R1, i1 = lib.rpcholqr_factor(plan, A, s, seed)
            torch.cuda.synchronize()
            assert i1.cpu().tolist() == [0, -1]
            assert torch.equal(Q, Q1) and torch.equal(R, R1)
        # graph capture + replay reproduces the same bits
        Qg, Rg, infog = lib.rpcholqr_batch_capture(batch, As, ss, seeds)
        lib.rpcholqr_batch_replay(batch)
        torch.cuda.synchronize()
        assert infog.cpu().view(-1, 2)[:, 0].eq(0).all()
        for Q, R, q, r in zip(Qs, Rs, Qg, Rg):
            assert torch.equal(Q, q) and torch.equal(R, r)
        lib.rpcholqr_batch_replay(batch)    # a second replay
        torch.cuda.synchronize()
        for Q, q in zip(Qs, Qg):
            assert torch.equal(Q, q)
    finally:
        batch.close()
        plan.close()


def test_batched_matches_oracle_and_autotune(lib, oracle_mod):
    As, ss, seeds = _make_batch()
    batch = lib.rpcholqr_batch_create(0, 1 << 17, 128, 384, slots=8)
    try:
        slots, ms = lib.rpcholqr_batch_autotune(batch, As, ss, seeds, reps=1)
        assert slots in (1, 2, 4, 8) and ms > 0
        Qs, Rs, info = lib.rpcholqr_batch_factor(batch, As, ss, seeds)
        torch.cuda.synchronize()
        for A, s, seed, Q, R in list(zip(As, ss, seeds, Qs, Rs))[:6]:
            Ah = A.cpu().numpy()
            o = oracle_mod.rpcholqr(Ah, s, seed)
            assert o["status"] == 0
            Rh = R.cpu().numpy()
            assert np.linalg.norm(Rh - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
            assert oracle_mod.orth_error(Q.cpu().numpy()) <= 10 * oracle_mod.orth_error(o["Q"]) + 1e-16
    finally:
        batch.close()


def test_batched_reports_per_matrix_status(lib):
    As, ss, seeds = _make_batch()
    bad = As[3].clone()
    bad[17, 5] = float("nan")
    As[3] = bad
    batch = lib.rpcholqr_batch_create(0, 1 << 17, 128, 384, slots=2)
    try:
        _, _, info = lib.rpcholqr_batch_factor(batch, As, ss, seeds)
        st = info.cpu().view(-1, 2)[:, 0].tolist()
        assert st[3] == lib.ERR_NONFINITE
        assert all(v == 0 for i, v in enumerate(st) if i != 3)
    finally:
        batch.close()
