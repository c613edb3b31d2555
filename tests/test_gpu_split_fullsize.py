"""SPLIT64 against the FP64 oracle at the sizes where the split kernels take their full-size branches.

At m = 2^20, n = 128 (the rpCholesky-QR workload of Section 5's shape, scaled up):
  * the 32-column FP64 row solves run two CTAs per SM over 256-row panels, 77,824 rows per wave, so
    every CTA's persistent panel loop takes several panels;
  * the split Gram gives each of its 76 row ranges about 13,800 rows, more than 64 exactness windows
    of 128 rows, so its int64 accumulator is flushed into the FP64 partial mid-range;
  * pass 2 streams A1 through the warp-specialised split product over 8,192 row tiles.
At m = 2^22, n = 256 (kappa = 1e12) pass 1 is the left-looking 64-column blocked solve with windowed
split updates (K up to 192) and the Gram and pass 2 cover several 64-column tiles.

Gates (the same as the smaller parity tests): R within 1e-12 relative; Q within max(1e-10, 10x the
oracle's own reversed-summation floor) for kappa <= 1e8; orthogonality and residual within 10x of the
oracle's and orthogonality <= 1e-13; the split Gram of the oracle's A1 within 4e-15 of the oracle's
Gram of the same A1, norm-wise and entry by entry (relative to ||G||).
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda", 0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def nrm2(x):
    return float(np.linalg.norm(x, 2))


@pytest.fixture(scope="module")
def headline(oracle_mod):
    """A = U diag(sigma) V^T, 2^20 x 128, kappa = 1e8, and the oracle's rpCholesky-QR of it (s = 3n)."""
    m, n, s, kappa, seed = 1 << 20, 128, 384, 1e8, 1
    A = inputs.usv(m, n, kappa, 20240620)
    o = oracle_mod.rpcholqr(A, s, seed, intermediates=True)
    assert o["status"] == 0
    return dict(A=A, o=o, m=m, n=n, s=s, kappa=kappa, seed=seed)


@pytest.fixture(scope="module")
def splan_full(lib):
    p = lib.rpcholqr_plan_create(0, 1 << 20, 128, 384, mode=lib.SPLIT64)
    yield p
    p.close()


def test_split_factor_full_size_against_oracle(lib, oracle_mod, headline, splan_full):
    A, o, s, seed = headline["A"], headline["o"], headline["s"], headline["seed"]
    Q, R, info = lib.rpcholqr_factor(splan_full, cu(A), s, seed)
    assert info.cpu().tolist() == [0, -1]
    assert not lib.rpcholqr_plan_split_pass2_fp64(splan_full)    # the tensor-core pass 2 ran
    Qh, Rh = host(Q), host(R)
    del Q
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, seed, variant=1)["Q"])
    assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)
    orth, orth_o = oracle_mod.orth_error_fast(Qh), oracle_mod.orth_error_fast(o["Q"])
    assert orth <= 1e-13 and orth <= 10 * orth_o
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])


def test_split_gram_window_flush_against_oracle(lib, oracle_mod, headline, splan_full):
    # 76 row ranges of ~13,800 rows: each range flushes its int64 window sums into FP64 mid-range
    A1 = headline["o"]["A1"]
    G, info = lib.rpcholqr_ozaki_gram(splan_full, cu(A1))
    assert int(info[0]) == 0
    Gh = host(G)
    ref = oracle_mod.gram(A1)
    g = nrm2(ref)
    assert np.array_equal(Gh, Gh.T)
    assert nrm2(Gh - ref) <= 4e-15 * g
    assert np.max(np.abs(Gh - ref)) <= 4e-15 * g


def test_split_factor_deterministic_full_size(lib, headline, splan_full):
    Ad = cu(headline["A"])
    Q1, R1, _ = lib.rpcholqr_factor(splan_full, Ad, headline["s"], 3)
    Q2, R2, info = lib.rpcholqr_factor(splan_full, Ad, headline["s"], 3)
    assert info.cpu().tolist() == [0, -1]
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


def test_split_factor_precision_config_against_oracle(lib, oracle_mod):
    # m = 2^22, n = 256, s = 3n, kappa = 1e12 (Q is determined only to ~u kappa: R, orthogonality and
    # residual are gated)
    m, n, s, kappa, seed = 1 << 22, 256, 768, 1e12, 2
    A = inputs.usv(m, n, kappa, 20240621)
    plan = lib.rpcholqr_plan_create(0, m, n, s, mode=lib.SPLIT64)
    try:
        Q, R, info = lib.rpcholqr_factor(plan, cu(A), s, seed)
        assert info.cpu().tolist() == [0, -1]
        Qh, Rh = host(Q), host(R)
        del Q
    finally:
        plan.close()
    torch.cuda.empty_cache()
    o = oracle_mod.rpcholqr(A, s, seed)
    assert o["status"] == 0
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    orth, orth_o = oracle_mod.orth_error_fast(Qh), oracle_mod.orth_error_fast(o["Q"])
    assert orth <= 1e-13 and orth <= 10 * orth_o
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])
