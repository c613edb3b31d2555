"""GPU tests of rpcholqr_factor_batched: many independent matrices in one persistent kernel launch.

The batched kernel runs, per matrix, the same device functions in the same arithmetic order as a single
rpcholqr_factor call on an FP64 plan with the same limits (sample, Householder R_s, pass-1 parts = the
single call's CTAs with their Gram partials summed in the same order, Cholesky, R = R1 R_s, pass 2).  So:
  * every matrix's Q and R are bit-identical to the single call's, and so are the statuses;
  * a matrix's results do not depend on what else is in the batch or in which order;
  * the results match the FP64 oracle under the parity gates of the single calls.
Failures are made on the host (a NaN in one matrix, a shape that does not fit the plan, a one-poll spin
limit); each is reported in that matrix's own status word.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

SHAPES = [(4096, 8), (30011, 128), (5000, 16), (70001, 64), (8192, 32), (12000, 100), (4500, 8),
          (20000, 50), (4096, 128), (9000, 1), (100000, 16), (6000, 77), (300, 33), (129, 40)]
MAX_M, MAX_N, MAX_S = 1 << 17, 128, 384


def _make(shapes=SHAPES, kappa_cycle=14, seed0=40):
    As, ss, seeds = [], [], []
    for i, (m, n) in enumerate(shapes):
        As.append(torch.from_numpy(inputs.usv(m, n, 10.0 ** (i % kappa_cycle), seed0 + i)).to(DEV))
        ss.append(min(3 * n, m))
        seeds.append(1000 + i)
    return As, ss, seeds


@pytest.fixture(scope="module")
def fplan(lib):
    p = lib.rpcholqr_plan_create(0, MAX_M, MAX_N, MAX_S, mode=lib.FP64)
    yield p
    p.close()


@pytest.fixture(scope="module")
def bplan(lib):
    p = lib.rpcholqr_plan_create(0, MAX_M, MAX_N, MAX_S, mode=lib.FP64)
    lib.rpcholqr_plan_set_option(p, lib.OPT_BATCH_CAPACITY, 64)
    yield p
    p.close()


def _status(info):
    return [tuple(x) for x in info.cpu().view(-1, 2).tolist()]


def test_batched_is_bit_identical_to_single_calls(lib, fplan, bplan):
    As, ss, seeds = _make()
    Qs, Rs, info, _ = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    torch.cuda.synchronize()
    assert _status(info) == [(0, -1)] * len(As)
    for A, s, seed, Q, R in zip(As, ss, seeds, Qs, Rs):
        Q1, R1, info1 = lib.rpcholqr_factor(fplan, A, s, seed)
        assert info1.cpu().tolist() == [0, -1]
        assert torch.equal(Q, Q1) and torch.equal(R, R1), (A.shape, s)


def test_batched_results_do_not_depend_on_the_batch(lib, bplan):
    As, ss, seeds = _make()
    Qs, Rs, _, _ = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    perm = list(reversed(range(len(As))))[::2] + [3, 3]       # a reordered subset with a repeat
    Qp, Rp, info, _ = lib.rpcholqr_factor_batched(bplan, [As[i] for i in perm], [ss[i] for i in perm],
                                                  [seeds[i] for i in perm])
    torch.cuda.synchronize()
    assert all(st == (0, -1) for st in _status(info))
    for k, i in enumerate(perm):
        assert torch.equal(Qp[k], Qs[i]) and torch.equal(Rp[k], Rs[i])


@pytest.mark.parametrize("idx", [1, 5, 7, 11])
def test_batched_matches_oracle(lib, oracle_mod, bplan, idx):
    As, ss, seeds = _make()
    Qs, Rs, info, _ = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    torch.cuda.synchronize()
    A = As[idx].cpu().numpy()
    o = oracle_mod.rpcholqr(A, ss[idx], seeds[idx])
    assert o["status"] == 0
    Qh, Rh = Qs[idx].cpu().numpy(), Rs[idx].cpu().numpy()
    assert np.linalg.norm(Rh - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
    assert oracle_mod.orth_error(Qh) <= 10 * oracle_mod.orth_error(o["Q"])
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])


def test_batched_reports_per_matrix_errors(lib, oracle_mod, fplan, bplan):
    As, ss, seeds = _make(SHAPES[:6])
    # a NaN outside the sample of matrix 2, an infinity inside the sample of matrix 4
    A2 = As[2].cpu().numpy()
    idx2 = set(oracle_mod.sample_indices(seeds[2], A2.shape[0], ss[2]).tolist())
    A2[next(r for r in range(A2.shape[0]) if r not in idx2), 3] = np.nan
    As[2] = torch.from_numpy(A2).to(DEV)
    A4 = As[4].cpu().numpy()
    A4[int(oracle_mod.sample_indices(seeds[4], A4.shape[0], ss[4])[7]), 0] = np.inf
    As[4] = torch.from_numpy(A4).to(DEV)
    # matrix 0: s < n does not fit; matrix 5: wider than the plan
    ss[0] = 4
    As[5] = torch.from_numpy(inputs.usv(3000, 130, 10.0, 9)).to(DEV)
    ss[5] = 390
    Qs, Rs, info, _ = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    st = _status(info)
    assert st[0][0] == lib.ERR_ARG and st[5][0] == lib.ERR_ARG
    assert st[2][0] == lib.ERR_NONFINITE and st[4][0] == lib.ERR_NONFINITE
    assert st[1] == (0, -1) and st[3] == (0, -1)
    Q1, R1, _ = lib.rpcholqr_factor(fplan, As[3], ss[3], seeds[3])
    assert torch.equal(Qs[3], Q1) and torch.equal(Rs[3], R1)


def test_batched_graph_capture_and_replay(lib, bplan):
    As, ss, seeds = _make()
    Qs, Rs, info, arrays = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    torch.cuda.synchronize()
    Q0 = [q.clone() for q in Qs]
    R0 = [r.clone() for r in Rs]
    for q in Qs:
        q.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            lib.rpcholqr_factor_batched(bplan, As, ss, seeds, Qs=Qs, Rs=Rs, info=info, stream=s, arrays=arrays)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert _status(info) == [(0, -1)] * len(As)
        assert all(torch.equal(a, b) for a, b in zip(Qs, Q0)) and all(torch.equal(a, b) for a, b in zip(Rs, R0))


def test_batched_one_poll_spin_limit_times_out_then_recovers(lib, bplan):
    As, ss, seeds = _make()
    Qs, Rs, info, arrays = lib.rpcholqr_factor_batched(bplan, As, ss, seeds)
    torch.cuda.synchronize()
    Q0 = [q.clone() for q in Qs]
    lib.rpcholqr_plan_set_option(bplan, lib.OPT_SPIN_LIMIT, 1)
    try:
        lib.rpcholqr_factor_batched(bplan, As, ss, seeds, Qs=Qs, Rs=Rs, info=info, arrays=arrays)
        st = [x[0] for x in _status(info)]
        # a dependency that is not complete at the first poll gives up; nothing else can go wrong
        assert set(st) <= {0, lib.ERR_TIMEOUT} and lib.ERR_TIMEOUT in st
    finally:
        lib.rpcholqr_plan_set_option(bplan, lib.OPT_SPIN_LIMIT, 1 << 24)
    lib.rpcholqr_factor_batched(bplan, As, ss, seeds, Qs=Qs, Rs=Rs, info=info, arrays=arrays)
    torch.cuda.synchronize()
    assert _status(info) == [(0, -1)] * len(As)
    assert all(torch.equal(a, b) for a, b in zip(Qs, Q0))


def test_batched_rejects_unsupported_plans(lib):
    A = [torch.from_numpy(inputs.usv(2000, 8, 10.0, 1)).to(DEV)]
    for mode, max_n in ((lib.SPLIT64, 64), (lib.FP64, 256)):
        p = lib.rpcholqr_plan_create(0, 4096, max_n, 3 * max_n, mode=mode)
        try:
            with pytest.raises(lib.RpcholqrError) as e:
                lib.rpcholqr_factor_batched(p, A, [24], [1])
            assert e.value.code == lib.ERR_UNSUPPORTED
        finally:
            p.close()
