"""GPU tests of the FP32 mode (float A, Q, R; FP64 sketch QR and Cholesky; FP32 passes).

The paper works in double precision only; this mode serves single-precision Krylov / LOBPCG data.
Gates (u32 = 2^-24): ||Q^T Q - I||_2 <= 1e-5 and ||A - QR||_2 / ||A||_2 <= 1e-5 up to kappa = 1e5
(the FP32 target), and agreement with the FP64 oracle on the same float values within the first-order
perturbation bound of a QR factor, max(1e-5, 50 u32 kappa(A)) (kappa times a backward error of a few
dozen u32).
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
DEV = torch.device("cuda", 0)


def host64(t):
    return t.detach().cpu().numpy().astype(np.float64)


def status(info):
    return tuple(int(x) for x in info.cpu().tolist())


def nrm2(x):
    return float(np.linalg.norm(x, 2))


@pytest.fixture(scope="module")
def fplan(lib):
    p = lib.rpcholqr_plan_create(0, 1 << 20, 512, 1536, mode=lib.FP32)
    yield p
    p.close()


def a32(m, n, kappa, seed):
    A = inputs.usv(m, n, kappa, seed).astype(np.float32)
    return A, A.astype(np.float64)     # the oracle factors exactly the float values


@pytest.mark.parametrize("m,n,kappa", [(20011, 50, 1.0), (30000, 128, 1e2), (20000, 128, 1e5),
                                       (12000, 256, 1e5), (9000, 300, 1e3), (4096, 7, 10.0),
                                       (16384, 512, 1e4), (1000, 33, 1e5)])
def test_fp32_factor_matches_oracle(lib, oracle_mod, fplan, m, n, kappa):
    A32, A64 = a32(m, n, kappa, 1300 + n)
    s = 3 * n
    Q, R, info = lib.rpcholqr_factor_f32(fplan, torch.from_numpy(A32).to(DEV), s, 5)
    assert status(info) == (0, -1)
    o = oracle_mod.rpcholqr(A64, s, 5)
    assert o["status"] == 0
    Qh, Rh = host64(Q), host64(R)
    assert np.array_equal(np.tril(Rh, -1), np.zeros((n, n)))
    assert np.all(np.diag(Rh) > 0)
    orth = oracle_mod.orth_error_fast(Qh)
    res = oracle_mod.residual(A64, Qh, Rh)
    assert orth <= 1e-5, orth
    assert res <= 1e-5, res
    tol = max(1e-5, 50 * U32 * kappa)
    assert nrm2(Rh - o["R"]) <= tol * nrm2(o["R"])
    assert nrm2(Qh - o["Q"]) <= tol


def test_fp32_nonfinite(lib, oracle_mod, fplan):
    A32, _ = a32(9000, 100, 10.0, 5)
    idx = set(oracle_mod.sample_indices(3, 9000, 300).tolist())
    A32[next(i for i in range(9000) if i not in idx), 77] = np.nan
    _, _, info = lib.rpcholqr_factor_f32(fplan, torch.from_numpy(A32).to(DEV), 300, 3)
    assert status(info)[0] == lib.ERR_NONFINITE


def test_fp32_deterministic_and_ld(lib, fplan):
    A32, _ = a32(30000, 96, 1e3, 8)
    A = torch.from_numpy(A32).to(DEV)
    Q1, R1, _ = lib.rpcholqr_factor_f32(fplan, A, 288, 11)
    Q2, R2, _ = lib.rpcholqr_factor_f32(fplan, A, 288, 11)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)
    # padded leading dimensions give the same bits
    Ap = torch.zeros((30000, 100), dtype=torch.float32, device=DEV)
    Ap[:, :96] = A
    Qp = torch.zeros((30000, 101), dtype=torch.float32, device=DEV)
    Q3, R3, info = lib.rpcholqr_factor_f32(fplan, Ap[:, :96], 288, 11, Q=Qp[:, :96])
    assert status(info) == (0, -1)
    assert torch.equal(Q3, Q1) and torch.equal(R3, R1)


def test_fp32_mode_checks(lib, fplan):
    A = torch.zeros((1000, 10), dtype=torch.float64, device=DEV)
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_factor(fplan, A, 30, 1)          # FP64 entry point on an FP32 plan
    p64 = lib.rpcholqr_plan_create(0, 1000, 10, 30)
    try:
        with pytest.raises(lib.RpcholqrError):
            lib.rpcholqr_factor_f32(p64, A.float(), 30, 1)
    finally:
        p64.close()


@pytest.mark.slow
def test_fp32_full_size(lib):
    # m = 2^22, n = 256, kappa = 1e5 in FP32: the single-precision workload
    m, n, kappa = 1 << 22, 256, 1e5
    A = inputs.usv_torch(m, n, kappa, 20240621, device=DEV).float()
    plan = lib.rpcholqr_plan_create(0, m, n, 3 * n, mode=lib.FP32)
    try:
        Q, R, info = lib.rpcholqr_factor_f32(plan, A, 3 * n, 1)
        assert status(info) == (0, -1)
        Qd, Rd, Ad = Q.double(), R.double(), A.double()
        orth = float(torch.linalg.matrix_norm(Qd.T @ Qd - torch.eye(n, dtype=torch.float64, device=DEV), 2))
        DD = torch.zeros((n, n), dtype=torch.float64, device=DEV)
        AA = torch.zeros_like(DD)
        for i in range(0, m, 1 << 20):
            d = Ad[i:i + (1 << 20)] - Qd[i:i + (1 << 20)] @ Rd
            DD += d.T @ d
            AA += Ad[i:i + (1 << 20)].T @ Ad[i:i + (1 << 20)]
        res = float(torch.linalg.eigvalsh(DD)[-1].clamp(min=0).sqrt() / torch.linalg.eigvalsh(AA)[-1].sqrt())
        print(f"fp32 full size m={m} n={n} kappa={kappa:g}: orth {orth:.3e} residual {res:.3e}")
        assert orth <= 1e-5 and res <= 1e-5
    finally:
        plan.close()
