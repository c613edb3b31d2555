"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same inputs.

Tolerances (FP64 throughout, u = 2^-53):
  * sample indices: bit-exact (integer work);
  * R (n x n): ||R_gpu - R_orc||_2 / ||R||_2 <= 1e-12 at every kappa -- two valid roundings of the
    oracle itself agree to ~1e-15 here (test_oracle::test_two_roundings...);
  * Q: ||Q_gpu - Q_orc||_2 <= max(1e-10, 10 ||Q_orc - Q_orc'||_2) for kappa(A) <= 1e8, where
    Q_orc' is the oracle with every summation reversed.  Q is only determined to ~u kappa(A) by A
    (the QR factor's own conditioning), so below kappa ~ 1e4 the absolute 1e-10 binds, above it the
    measured floor does;
  * every kappa: ||Q^T Q - I|| and ||A - QR|| / ||A|| within 10x of the oracle's own values;
  * steps in isolation: backward errors at the u level (row solves) and Gram/Cholesky/product
    agreement at 1e-13 relative, all with the oracle's intermediate injected so errors do not compound.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
DEV = torch.device("cuda", 0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def status(info):
    return tuple(int(x) for x in info.cpu().tolist())


@pytest.fixture(scope="module")
def plan(lib):
    p = lib.rpcholqr_plan_create(0, 1 << 21, 128, 1536)
    yield p
    p.close()


def nrm2(x):
    return float(np.linalg.norm(x, 2))


# ---- a1 sample indices --------------------------------------------------------------------------
@pytest.mark.parametrize("m,s,seed,stream_id", [
    (1, 5, 1, 0), (7, 3, 2, 0), (10000, 150, 3, 0), (10007, 1281, 4, 0), (1 << 20, 384, 5, 0),
    (2**40 + 3, 777, 6, 0), (2**62 + 11, 64, 7, 9), (123457, 4099, 2**64 - 1, 2**63)])
def test_sample_indices_bit_exact(lib, oracle_mod, m, s, seed, stream_id):
    idx = lib.rpcholqr_sample_indices(seed, m, s, stream_id=stream_id, device=DEV)
    assert np.array_equal(host(idx), oracle_mod.sample_indices(seed, m, s, stream=stream_id))


# ---- a2 + a3 sample and Householder R_s ----------------------------------------------------------
@pytest.mark.parametrize("m,n,s,kappa", [(10007, 50, 150, 1e8), (5000, 128, 384, 1e12),
                                         (3001, 7, 70, 1.0), (4096, 1, 3, 1e3), (10000, 100, 1000, 1e16),
                                         (2000, 128, 128, 1e4)])
def test_sketch_r_matches_oracle(lib, oracle_mod, plan, m, n, s, kappa):
    A = inputs.usv(m, n, kappa, 100 + n)
    Rs, info = lib.rpcholqr_sketch_r(plan, cu(A), s, 17)
    assert status(info) == (0, -1)
    o = oracle_mod.rpcholqr(A, s, 17)
    Rs_o = o["Rs"]
    assert np.all(np.diag(host(Rs)) > 0)
    assert np.array_equal(np.tril(host(Rs), -1), np.zeros((n, n)))
    assert nrm2(host(Rs) - Rs_o) <= 1e-13 * nrm2(Rs_o)


# ---- a4 + a5 fused preconditioning pass and Gram -------------------------------------------------
@pytest.mark.parametrize("m,n,kappa", [(10007, 50, 1e3), (2049, 128, 1e8), (300, 16, 1e12),
                                       (129, 1, 1.0), (1000, 33, 1e5), (7777, 112, 1e16)])
def test_precondition_gram_matches_oracle(lib, oracle_mod, plan, m, n, kappa):
    A = inputs.usv(m, n, kappa, 200 + n)
    o = oracle_mod.rpcholqr(A, 3 * n, 21, intermediates=True)
    Rs = o["Rs"]
    A1, G, info = lib.rpcholqr_precondition_gram(plan, cu(A), cu(Rs))
    assert status(info)[0] == 0
    A1h, Gh = host(A1), host(G)
    # backward error of the m row solves (row-wise, Section 2.1): A1 Rs = A + E, |E| ~ u |A1||Rs|
    E = A1h @ Rs - A
    bound = (np.abs(A1h) @ np.abs(Rs))
    assert np.max(np.abs(E) / np.maximum(bound, 1e-300)) <= 4 * n * EPS
    # forward agreement where kappa(A) leaves it determined
    if kappa <= 1e5:
        assert nrm2(A1h - o["A1"]) <= 1e-13 * max(1.0, kappa / 1e2) * nrm2(o["A1"])
    # Gram of the GPU's own A1 against the oracle's Gram of the same A1
    G_o = oracle_mod.gram(A1h)
    assert np.array_equal(Gh, Gh.T)
    assert nrm2(Gh - G_o) <= 1e-13 * nrm2(G_o)


def test_precondition_flags_nonfinite(lib, plan):
    A = inputs.usv(5000, 20, 10.0, 3)
    A[4321, 7] = np.inf
    Rs = np.eye(20)
    _, _, info = lib.rpcholqr_precondition_gram(plan, cu(A), cu(Rs))
    assert status(info)[0] == lib.ERR_NONFINITE


# ---- a6 Cholesky --------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 5, 16, 50, 127, 128])
def test_cholesky_matches_oracle(lib, oracle_mod, plan, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((4 * n + 3, n))
    G = X.T @ X
    R1, info = lib.rpcholqr_cholesky(plan, cu(G))
    assert status(info) == (0, -1)
    R_o, st, _ = oracle_mod.cholesky_upper(G)
    assert st == 0
    assert nrm2(host(R1) - R_o) <= 1e-13 * nrm2(R_o)


def test_cholesky_not_spd_pivot(lib, plan):
    G = np.diag([4.0, 1.0, 9.0, -1.0, 2.0])
    _, info = lib.rpcholqr_cholesky(plan, cu(G))
    assert status(info) == (lib.ERR_NOT_SPD, 3)
    G = np.eye(6)
    G[2, 2] = np.nan
    _, info = lib.rpcholqr_cholesky(plan, cu(G))
    assert status(info) == (lib.ERR_NOT_SPD, 2)


# ---- a7 second pass (row solve) ---------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(10007, 50), (2048, 128), (257, 7), (130, 1)])
def test_solve_rows_matches_oracle(lib, oracle_mod, plan, m, n):
    rng = np.random.default_rng(m + n)
    X = rng.standard_normal((m, n))
    T = np.triu(rng.standard_normal((n, n)) * 0.3) + np.diag(1.0 + rng.random(n))
    Y, info = lib.rpcholqr_solve_rows(plan, cu(X), cu(T))
    assert status(info)[0] == 0
    Y_o = oracle_mod.trsm_rows(X, T)
    assert nrm2(host(Y) - Y_o) <= 1e-12 * nrm2(Y_o)
    # in place
    Xd = cu(X)
    Y2, _ = lib.rpcholqr_solve_rows(plan, Xd, cu(T), Y=Xd)
    assert np.array_equal(host(Y2), host(Y))


# ---- a8 R = R1 Rs ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 9, 64, 128])
def test_triu_mul_matches_oracle(lib, oracle_mod, n):
    rng = np.random.default_rng(n)
    a = np.triu(rng.standard_normal((n, n)))
    b = np.triu(rng.standard_normal((n, n)))
    R = lib.rpcholqr_triu_mul(cu(a), cu(b))
    torch.cuda.synchronize()
    ref = oracle_mod.triu_mul(a, b)
    assert np.max(np.abs(host(R) - ref)) <= 8 * n * EPS * np.max(np.abs(a) @ np.abs(b))


# ---- end to end --------------------------------------------------------------------------------------
def _check_against_oracle(lib, oracle_mod, plan, A, s, seed, kappa, fast_metrics=False):
    Q, R, info = lib.rpcholqr_factor(plan, cu(A), s, seed)
    st = status(info)
    o = oracle_mod.rpcholqr(A, s, seed)
    assert st[0] == o["status"] == 0, (st, o["status"])
    Qh, Rh = host(Q), host(R)
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    if kappa <= 1e8:
        floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, seed, variant=1)["Q"])
        assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)
    orth = oracle_mod.orth_error_fast(Qh) if fast_metrics else oracle_mod.orth_error(Qh)
    orth_o = oracle_mod.orth_error_fast(o["Q"]) if fast_metrics else oracle_mod.orth_error(o["Q"])
    assert orth <= 10 * orth_o
    if not fast_metrics:
        assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])
    return Qh, Rh, o


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e12, 1e16])
def test_factor_kappa_sweep(lib, oracle_mod, plan, kappa):
    m, n = 10007, 50
    A = inputs.usv(m, n, kappa, 300)
    _check_against_oracle(lib, oracle_mod, plan, A, 3 * n, 7, kappa)


def test_factor_small_config(lib, oracle_mod, plan):
    # m = 10,000, n = 50, s = 3n = 150, sigma log-spaced to 1e-8
    A = inputs.usv(10000, 50, 1e8, 20240617)
    _check_against_oracle(lib, oracle_mod, plan, A, 150, 1, 1e8)


@pytest.mark.parametrize("m,n,s", [(128, 128, 128), (500, 1, 1), (1000, 7, 21), (4099, 16, 48),
                                   (3333, 64, 640), (20000, 127, 381), (70001, 128, 1280),
                                   (999, 100, 999)])
def test_factor_shapes(lib, oracle_mod, plan, m, n, s):
    A = inputs.usv(m, n, 1e6, m + n)
    _check_against_oracle(lib, oracle_mod, plan, A, s, 3, 1e6)


def test_factor_orthonormal_input(lib, plan):
    u, _, _ = inputs.usv_factors(5000, 40, 1.0, 4)
    Q, R, info = lib.rpcholqr_factor(plan, cu(u), 120, 2)
    assert status(info)[0] == 0
    assert nrm2(host(R) - np.eye(40)) <= 1e-14
    assert nrm2(host(Q) - u) <= 1e-14


def test_factor_leading_dimensions(lib, oracle_mod, plan):
    A = inputs.usv(3000, 30, 1e4, 9)
    big = torch.zeros((3000, 37), dtype=torch.float64, device=DEV)
    big[:, :30] = cu(A)
    Aview = big[:, :30]
    Qbig = torch.full((3000, 41), 7.0, dtype=torch.float64, device=DEV)
    Q, R, info = lib.rpcholqr_factor(plan, Aview, 90, 5, Q=Qbig[:, :30])
    assert status(info)[0] == 0
    Q2, R2, _ = lib.rpcholqr_factor(plan, cu(A), 90, 5)
    assert torch.equal(Q, Q2) and torch.equal(R, R2)
    assert torch.all(Qbig[:, 30:] == 7.0)


def test_factor_deterministic_and_stream(lib, plan):
    A = cu(inputs.usv(50000, 128, 1e10, 8))
    Q1, R1, _ = lib.rpcholqr_factor(plan, A, 384, 11)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Q2, R2, info = lib.rpcholqr_factor(plan, A, 384, 11, stream=s)
    s.synchronize()
    assert status(info)[0] == 0
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


def test_factor_host_matches_device(lib, plan):
    A = inputs.usv(20011, 64, 1e6, 12)
    Qd, Rd, _ = lib.rpcholqr_factor(plan, cu(A), 192, 4)
    Ah = torch.from_numpy(A).pin_memory()
    Qh, Rh, st, piv = lib.rpcholqr_factor_host(plan, Ah, 192, 4)
    assert (st, piv) == (0, -1)
    assert np.array_equal(Qh.numpy(), host(Qd)) and np.array_equal(Rh.numpy(), host(Rd))


# ---- error paths (all made on the host) ------------------------------------------------------------
def test_factor_nonfinite_outside_sample(lib, oracle_mod, plan):
    A = inputs.usv(8000, 20, 10.0, 5)
    idx = set(oracle_mod.sample_indices(3, 8000, 60).tolist())
    r = next(i for i in range(8000) if i not in idx)
    A[r, 4] = np.nan
    _, _, info = lib.rpcholqr_factor(plan, cu(A), 60, 3)
    assert status(info)[0] == lib.ERR_NONFINITE


def test_factor_nonfinite_in_sample(lib, oracle_mod, plan):
    A = inputs.usv(8000, 20, 10.0, 5)
    A[int(oracle_mod.sample_indices(3, 8000, 60)[5]), 0] = -np.inf
    _, _, info = lib.rpcholqr_factor(plan, cu(A), 60, 3)
    assert status(info)[0] == lib.ERR_NONFINITE


def test_factor_coherent_gives_singular_sketch(lib, oracle_mod, plan):
    A = inputs.coherent_diag(50000, 30, 2)
    o = oracle_mod.rpcholqr(A, 90, 6)
    assert o["status"] == oracle_mod.ERR_SINGULAR_SKETCH
    _, _, info = lib.rpcholqr_factor(plan, cu(A), 90, 6)
    assert status(info)[0] == lib.ERR_SINGULAR_SKETCH


def test_factor_rejects_bad_shapes(lib, plan):
    A = cu(np.ones((100, 10)))
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_factor(plan, A, 9, 1)          # s < n
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_factor(plan, A, 101, 1)        # s > m
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_factor(plan, cu(np.ones((2000, 129))), 400, 1)   # n > plan max


def test_fp64_probe_reports_a_rate(lib):
    r = lib.rpcholqr_probe_fp64_mma(0, 512)
    assert 1e12 < r < 1e14


# ---- full size, in the launch configuration bench.py times ----------------------------------------
@pytest.mark.slow
def test_factor_full_size_against_oracle(lib, oracle_mod):
    # m = 2^20, n = 128, s = 3n, kappa = 1e8: the benchmark workload
    m, n, s, kappa = 1 << 20, 128, 384, 1e8
    A = inputs.usv(m, n, kappa, 20240619)
    plan = lib.rpcholqr_plan_create(0, m, n, 3 * 1280)
    try:
        _check_against_oracle(lib, oracle_mod, plan, A, s, 1, kappa, fast_metrics=True)
    finally:
        plan.close()


# ---- Cholesky-QR / Cholesky-QR2 (the comparison method of Section 5.3) -------------------------------
@pytest.mark.parametrize("m,n,kappa", [(10007, 50, 1e2), (20000, 128, 1e6), (3000, 7, 1e4)])
def test_cholqr2_matches_oracle(lib, oracle_mod, plan, m, n, kappa):
    # Cholesky-QR's factors depend on the rounding of A^T A (kappa(A)^2 u), so R is gated against the
    # oracle's own floor (every sum reversed) as well as the absolute 1e-12.
    A = inputs.usv(m, n, kappa, 900 + n)
    Q, R, info = lib.rpcholqr_cholqr2(plan, cu(A))
    assert status(info) == (0, -1)
    o = oracle_mod.cholqr2(A)
    o_rev = oracle_mod.cholqr2(A, variant=1)
    assert o["status"] == 0
    floor = nrm2(o["R"] - o_rev["R"])
    assert nrm2(host(R) - o["R"]) <= max(1e-12 * nrm2(o["R"]), 10 * floor)
    assert oracle_mod.orth_error(host(Q)) <= 10 * oracle_mod.orth_error(o["Q"]) + 1e-15
    Q1, R1, info1 = lib.rpcholqr_cholqr(plan, cu(A))
    o1 = oracle_mod.cholqr(A)
    floor1 = nrm2(o1["R"] - oracle_mod.cholqr(A, variant=1)["R"])
    assert status(info1) == (0, -1)
    assert nrm2(host(R1) - o1["R"]) <= max(1e-12 * nrm2(o1["R"]), 10 * floor1)


def test_cholqr2_breaks_down_where_rpcholqr_succeeds(lib, oracle_mod, plan):
    # kappa = 1e16: the Gram matrix is not numerically SPD (Section 1, Existing work)
    A = inputs.usv(20000, 64, 1e16, 33)
    _, _, info = lib.rpcholqr_cholqr2(plan, cu(A))
    assert status(info)[0] == lib.ERR_NOT_SPD
    assert oracle_mod.cholqr2(A)["status"] == oracle_mod.ERR_NOT_SPD
    Q, R, info = lib.rpcholqr_factor(plan, cu(A), 192, 1)
    assert status(info) == (0, -1)
    assert oracle_mod.orth_error(host(Q)) <= 1e-13


# ---- shifted Cholesky-QR3 (the remedy for Cholesky-QR2's breakdown cited in Section 1) ----------------
@pytest.mark.parametrize("m,n,kappa", [(3000, 40, 1e2), (3000, 40, 1e12), (20000, 128, 1e10), (6000, 200, 1e11)])
def test_scholqr3_matches_oracle(lib, oracle_mod, m, n, kappa):
    A = inputs.usv(m, n, kappa, 51 if n == 40 else 700 + n)
    plan = lib.rpcholqr_plan_create(0, m, n, 3 * n)
    try:
        Q, R, info = lib.rpcholqr_scholqr3(plan, cu(A))
        assert status(info) == (0, -1)
    finally:
        plan.close()
    o = oracle_mod.scholqr3(A)
    assert o["status"] == 0
    # the first stage's factor carries kappa(A)-level sensitivity: R is gated on the oracle's own floor
    floor = nrm2(o["R"] - oracle_mod.scholqr3(A, variant=1)["R"])
    assert nrm2(host(R) - o["R"]) <= max(1e-12 * nrm2(o["R"]), 10 * floor)
    assert oracle_mod.orth_error(host(Q)) <= 10 * oracle_mod.orth_error(o["Q"]) + 1e-15
    assert oracle_mod.residual(A, host(Q), host(R)) <= 10 * oracle_mod.residual(A, o["Q"], o["R"]) + 1e-16


def test_scholqr3_breaks_down_beyond_its_range(lib, oracle_mod):
    A = inputs.usv(3000, 40, 1e15, 51)
    plan = lib.rpcholqr_plan_create(0, 3000, 40, 120)
    try:
        _, _, info = lib.rpcholqr_scholqr3(plan, cu(A))
        assert status(info)[0] == lib.ERR_NOT_SPD
        Q, R, info = lib.rpcholqr_factor(plan, cu(A), 120, 1)
        assert status(info) == (0, -1)
        assert oracle_mod.orth_error(host(Q)) <= 1e-13
    finally:
        plan.close()
