"""GPU parity for wide panels (128 < n <= 2048): left-looking blocked solves over 64-column blocks, the
blocked FP64 Gram, the windowed split products (K > 128) and the tiled split Gram, in both modes.

Same gates as the narrow tests: R within 1e-12 of the oracle, Q within max(1e-10, 10x the oracle's
reversed-sum floor) for kappa <= 1e8, orthogonality and residual within 10x of the oracle's, and the
split mode at ||Q^T Q - I|| <= 1e-13.  The full-size cases (m = 2^22, n = 256 and m = 2^23, n = 512,
34 GB per copy of A) are checked through what the oracle can compute there (the sketch R_s) and
through properties that hold at any size (orthogonality, residual, agreement of the two modes).
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


def nrm2(x):
    return float(np.linalg.norm(x, 2))


def pow2_bound(v, axis):
    mx = np.max(np.abs(v), axis=axis)
    return np.where(mx > 0, 2.0 ** (np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 1), 0.0)


@pytest.fixture(scope="module")
def plans(lib):
    ps = {"fp64": lib.rpcholqr_plan_create(0, 40000, 512, 1536),
          "split": lib.rpcholqr_plan_create(0, 40000, 512, 1536, mode=lib.SPLIT64)}
    yield ps
    for p in ps.values():
        p.close()


# ---- end to end against the oracle ------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("m,n,kappa", [(20011, 192, 1e8), (30000, 256, 1e12), (12000, 300, 1e4),
                                       (16384, 512, 1e8), (25000, 256, 1e16), (2000, 129, 1e6)])
def test_wide_factor_matches_oracle(lib, oracle_mod, plans, mode, m, n, kappa):
    A = inputs.usv(m, n, kappa, 1100 + n)
    s = 3 * n
    Q, R, info = lib.rpcholqr_factor(plans[mode], cu(A), s, 9)
    assert status(info) == (0, -1)
    o = oracle_mod.rpcholqr(A, s, 9)
    assert o["status"] == 0
    Qh, Rh = host(Q), host(R)
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    fast = n > 300
    orth = oracle_mod.orth_error_fast(Qh) if fast else oracle_mod.orth_error(Qh)
    orth_o = oracle_mod.orth_error_fast(o["Q"]) if fast else oracle_mod.orth_error(o["Q"])
    assert orth <= 10 * orth_o
    if mode == "split":
        assert orth <= 1e-13
    if not fast:
        assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])
    if kappa <= 1e8:
        floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, 9, variant=1)["Q"])
        assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)


# The stage images of the wide split passes: by default every row (the first pass and the Gram one launch
# over all rows); with OPT_IMAGE_ROWS set below m they and the second pass run row chunk by row chunk
# (ragged last chunks here).  Both match the oracle; the option reads back, and a plan that is not
# SPLIT64 above 128 columns refuses it.
@pytest.mark.parametrize("m,n,kappa", [(20011, 576, 1e8), (9001, 448, 1e14)])
def test_split_image_rows_option(lib, oracle_mod, m, n, kappa):
    A = inputs.usv(m, n, kappa, 1300 + n)
    s = 3 * n
    o = oracle_mod.rpcholqr(A, s, 5)
    assert o["status"] == 0
    plan = lib.rpcholqr_plan_create(0, m, n, s, mode=lib.SPLIT64)
    try:
        all_rows = (m + 127) // 128 * 128
        assert lib.rpcholqr_plan_get_option(plan, lib.OPT_IMAGE_ROWS) == all_rows
        for rows in (0, 4000, 128 * 17):
            lib.rpcholqr_plan_set_option(plan, lib.OPT_IMAGE_ROWS, rows)
            assert lib.rpcholqr_plan_get_option(plan, lib.OPT_IMAGE_ROWS) == (all_rows if rows == 0 else
                                                                             (rows + 127) // 128 * 128)
            Q, R, info = lib.rpcholqr_factor(plan, cu(A), s, 5)
            assert status(info) == (0, -1)
            Qh, Rh = host(Q), host(R)
            assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
            orth = oracle_mod.orth_error_fast(Qh)
            assert orth <= 1e-13 and orth <= 10 * oracle_mod.orth_error_fast(o["Q"])
            if kappa <= 1e8:
                floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, 5, variant=1)["Q"])
                assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)
        with pytest.raises(lib.RpcholqrError):
            lib.rpcholqr_plan_set_option(plan, lib.OPT_IMAGE_ROWS, -1)
    finally:
        plan.close()
    narrow = lib.rpcholqr_plan_create(0, 4096, 128, 384, mode=lib.SPLIT64)
    try:
        with pytest.raises(lib.RpcholqrError) as e:
            lib.rpcholqr_plan_set_option(narrow, lib.OPT_IMAGE_ROWS, 4096)
        assert e.value.code == lib.ERR_UNSUPPORTED
    finally:
        narrow.close()


@pytest.fixture(scope="module")
def xplans(lib):
    ps = {"fp64": lib.rpcholqr_plan_create(0, 12000, 2048, 6144),
          "split": lib.rpcholqr_plan_create(0, 12000, 2048, 6144, mode=lib.SPLIT64)}
    yield ps
    for p in ps.values():
        p.close()


_XW_CACHE = {}


def _xw_oracle(oracle_mod, m, n, kappa, s):
    """Input and oracle results of one extra-wide case, computed once for both modes."""
    key = (m, n, kappa, s)
    if key not in _XW_CACHE:
        A = inputs.usv(m, n, kappa, 1300 + n)
        o = oracle_mod.rpcholqr(A, s, 4)
        assert o["status"] == 0
        floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, 4, variant=1)["Q"]) if kappa <= 1e8 else None
        _XW_CACHE[key] = (A, o["R"], o["Q"], oracle_mod.orth_error_fast(o["Q"]), floor)
    return _XW_CACHE[key]


@pytest.mark.parametrize("m,n,kappa", [(12000, 1000, 1e8), (10007, 2048, 1e10), (8000, 777, 1e14)])
@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_extra_wide_factor_matches_oracle(lib, oracle_mod, xplans, mode, m, n, kappa):
    # n > 512: R1^{-1} by the FP64 row solve of the identity, products with K up to 2048, Gram partials
    # capped by rows; the same gates as above
    s = 3 * n if 3 * n <= 6144 else 6144
    A, R_o, Q_o, orth_o, floor = _xw_oracle(oracle_mod, m, n, kappa, s)
    Q, R, info = lib.rpcholqr_factor(xplans[mode], cu(A), s, 4)
    assert status(info) == (0, -1)
    Qh, Rh = host(Q), host(R)
    assert nrm2(Rh - R_o) <= 1e-12 * nrm2(R_o)
    orth = oracle_mod.orth_error_fast(Qh)
    assert orth <= 10 * orth_o
    if mode == "split":
        assert orth <= 1e-13
    if floor is not None:
        assert nrm2(Qh - Q_o) <= max(1e-10, 10 * floor)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_wide_factor_nonfinite_in_late_block(lib, oracle_mod, plans, mode):
    # a NaN in column 450 (block 7) of a row outside the sample: caught by that block's row pass
    m, n, s = 9000, 480, 1440
    A = inputs.usv(m, n, 10.0, 5)
    idx = set(oracle_mod.sample_indices(3, m, s).tolist())
    A[next(i for i in range(m) if i not in idx), 450] = np.nan
    _, _, info = lib.rpcholqr_factor(plans[mode], cu(A), s, 3)
    assert status(info)[0] == lib.ERR_NONFINITE


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_wide_factor_deterministic(lib, plans, mode):
    A = cu(inputs.usv(30000, 320, 1e10, 8))
    Q1, R1, _ = lib.rpcholqr_factor(plans[mode], A, 960, 11)
    Q2, R2, _ = lib.rpcholqr_factor(plans[mode], A, 960, 11)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


# ---- steps in isolation ------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,kappa", [(10007, 256, 1e3), (4099, 200, 1e12), (20000, 512, 1e6)])
def test_wide_precondition_gram(lib, oracle_mod, plans, m, n, kappa):
    A = inputs.usv(m, n, kappa, 1200 + n)
    o = oracle_mod.rpcholqr(A, 3 * n, 21, intermediates=True)
    Rs = o["Rs"]
    A1, G, info = lib.rpcholqr_precondition_gram(plans["fp64"], cu(A), cu(Rs))
    assert status(info)[0] == 0
    A1h, Gh = host(A1), host(G)
    E = A1h @ Rs - A
    bound = np.abs(A1h) @ np.abs(Rs)
    assert np.max(np.abs(E) / np.maximum(bound, 1e-300)) <= 4 * n * EPS
    G_o = oracle_mod.gram(A1h)
    assert np.array_equal(Gh, Gh.T)
    assert nrm2(Gh - G_o) <= 1e-13 * nrm2(G_o)


@pytest.mark.parametrize("m,n", [(10007, 300), (2048, 512), (1000, 129), (4096, 192)])
def test_wide_solve_rows(lib, oracle_mod, plans, m, n):
    rng = np.random.default_rng(m + n)
    X = rng.standard_normal((m, n))
    T = np.triu(rng.standard_normal((n, n)) * 0.3 / np.sqrt(n)) + np.diag(1.0 + rng.random(n))
    Y, info = lib.rpcholqr_solve_rows(plans["fp64"], cu(X), cu(T))
    assert status(info)[0] == 0
    Y_o = oracle_mod.trsm_rows(X, T)
    assert nrm2(host(Y) - Y_o) <= 1e-12 * nrm2(Y_o)
    Xd = cu(X)
    Y2, _ = lib.rpcholqr_solve_rows(plans["fp64"], Xd, cu(T), Y=Xd)
    assert np.array_equal(host(Y2), host(Y))


@pytest.mark.parametrize("n", [129, 200, 384, 512])
def test_wide_cholesky(lib, oracle_mod, plans, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((4 * n + 3, n))
    G = X.T @ X
    R1, info = lib.rpcholqr_cholesky(plans["fp64"], cu(G))
    assert status(info) == (0, -1)
    R_o, st, _ = oracle_mod.cholesky_upper(G)
    assert st == 0
    assert nrm2(host(R1) - R_o) <= 1e-13 * nrm2(R_o)


def test_wide_cholesky_not_spd_pivot(lib, plans):
    G = np.eye(300)
    G[257, 257] = -1.0
    _, info = lib.rpcholqr_cholesky(plans["fp64"], cu(G))
    assert status(info) == (lib.ERR_NOT_SPD, 257)


def test_wide_triu_mul(lib, oracle_mod):
    n = 512
    rng = np.random.default_rng(n)
    a = np.triu(rng.standard_normal((n, n)))
    b = np.triu(rng.standard_normal((n, n)))
    R = lib.rpcholqr_triu_mul(cu(a), cu(b))
    torch.cuda.synchronize()
    ref = oracle_mod.triu_mul(a, b)
    assert np.max(np.abs(host(R) - ref)) <= 8 * n * EPS * np.max(np.abs(a) @ np.abs(b))


@pytest.mark.parametrize("m,K,N", [(1000, 300, 200), (4099, 512, 512), (300, 129, 64), (20000, 256, 100)])
def test_wide_ozaki_gemm(lib, plans, m, K, N):
    rng = np.random.default_rng(m + K + N)
    X = rng.standard_normal((m, K)) * (10.0 ** rng.uniform(-6, 6, size=(m, 1)))
    Y = np.triu(rng.standard_normal((K, N)) * (10.0 ** rng.uniform(-3, 3, size=(1, N))))
    C, info = lib.rpcholqr_ozaki_gemm(plans["split"], cu(X), cu(Y))
    assert int(info[0]) == 0
    ref = X @ Y
    scale = pow2_bound(X, 1)[:, None] * pow2_bound(Y, 0)[None, :]
    assert np.max(np.abs(host(C) - ref) / np.maximum(scale, 1e-300)) <= 8 * K * EPS


def test_wide_ozaki_gemm_exact_on_small_integers(lib, plans):
    rng = np.random.default_rng(4)
    X = rng.integers(-1000, 1000, size=(777, 480)).astype(np.float64)
    Y = rng.integers(-1000, 1000, size=(480, 200)).astype(np.float64)
    C, info = lib.rpcholqr_ozaki_gemm(plans["split"], cu(X), cu(Y))
    assert int(info[0]) == 0
    assert np.array_equal(host(C), X @ Y)


@pytest.mark.parametrize("m,n", [(10007, 256), (4099, 300), (20000, 512), (3000, 129), (40000, 192)])
def test_wide_ozaki_gram(lib, oracle_mod, plans, m, n):
    A = inputs.usv(m, n, 1e3, m + n)
    A1 = oracle_mod.rpcholqr(A, 3 * n, 1, intermediates=True)["A1"]
    G, info = lib.rpcholqr_ozaki_gram(plans["split"], cu(A1))
    assert int(info[0]) == 0
    ref = oracle_mod.gram(A1)
    Gh = host(G)
    assert np.array_equal(Gh, Gh.T)
    assert nrm2(Gh - ref) <= 4e-15 * nrm2(ref)


def test_wide_cholqr2(lib, oracle_mod, plans):
    A = inputs.usv(20000, 256, 1e5, 77)
    Q, R, info = lib.rpcholqr_cholqr2(plans["fp64"], cu(A))
    assert status(info) == (0, -1)
    o = oracle_mod.cholqr2(A)
    floor = nrm2(o["R"] - oracle_mod.cholqr2(A, variant=1)["R"])
    assert nrm2(host(R) - o["R"]) <= max(1e-12 * nrm2(o["R"]), 10 * floor)
    assert oracle_mod.orth_error(host(Q)) <= 10 * oracle_mod.orth_error(o["Q"]) + 1e-15


# ---- full sizes -------------------------------------------------------------------------------------
def _gpu_orth(Q):
    n = Q.shape[1]
    return float(torch.linalg.matrix_norm(Q.T @ Q - torch.eye(n, dtype=Q.dtype, device=Q.device), 2))


def _gpu_residual(A, Q, R, rows=1 << 20):
    # ||A - QR||_2 / ||A||_2 through the n x n Gram matrices of row chunks (no m x n temporaries)
    n = A.shape[1]
    DD = torch.zeros((n, n), dtype=A.dtype, device=A.device)
    AA = torch.zeros_like(DD)
    for i in range(0, A.shape[0], rows):
        a = A[i:i + rows]
        d = a - Q[i:i + rows] @ R
        DD += d.T @ d
        AA += a.T @ a
    return float(torch.linalg.eigvalsh(DD)[-1].clamp(min=0).sqrt() / torch.linalg.eigvalsh(AA)[-1].sqrt())


@pytest.mark.slow
@pytest.mark.parametrize("m,n,kappa", [(1 << 22, 256, 1e12), (1 << 23, 512, 1e18)])
def test_wide_full_size(lib, oracle_mod, m, n, kappa):
    s = 3 * n
    A = inputs.usv_torch(m, n, kappa, 20240620 + n, device=DEV)
    # the sketch R_s, which the oracle computes from the s sampled rows alone
    idx = oracle_mod.sample_indices(1, m, s)
    rows = host(A[torch.from_numpy(idx).to(DEV)])
    Rs_o = oracle_mod.householder_r(np.sqrt(m / s) * rows)[0]
    results = {}
    for mode in ("fp64", "split"):
        plan = lib.rpcholqr_plan_create(0, m, n, s, mode=lib.SPLIT64 if mode == "split" else lib.FP64)
        try:
            Rs, info = lib.rpcholqr_sketch_r(plan, A, s, 1)
            assert status(info) == (0, -1)
            assert nrm2(host(Rs) - Rs_o) <= 1e-13 * nrm2(Rs_o)
            Q, R, info = lib.rpcholqr_factor(plan, A, s, 1)
            assert status(info) == (0, -1)
            results[mode] = (_gpu_orth(Q), _gpu_residual(A, Q, R), host(R))
            del Q
        finally:
            plan.close()
        torch.cuda.empty_cache()
    # Section 5 (experiments with c = 3n samples, n up to 2000): deviation from orthonormality below
    # 1e-12 and residuals near 1e-16 even for numerically singular A; the split mode within 10x of FP64
    for mode, (orth, res, _) in results.items():
        print(f"full size m={m} n={n} kappa={kappa:g} {mode}: orth {orth:.3e} residual {res:.3e}")
        assert orth <= 1e-12, (mode, orth)
        assert res <= 1e-14, (mode, res)
    assert results["split"][0] <= 10 * results["fp64"][0]
    R64, Rsp = results["fp64"][2], results["split"][2]
    assert nrm2(Rsp - R64) <= 1e-12 * nrm2(R64)
