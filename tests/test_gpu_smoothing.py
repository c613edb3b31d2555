"""GPU parity of the smoothing F = F_T D (two-pass fast Walsh-Hadamard transform) against the oracle's
direct definition, and of rpCholesky-QR with smoothing on the maximally coherent inputs of Section
5.1 (Eq. e_ErrorRange), which fail without it.

Tolerance of the smoothed sample: the oracle forms each sampled entry as a plain sum over the m rows
(rounding error below m u sum|a_i|), the GPU by p = log2 m' butterfly stages (below p u sum|a_i|), so
|A_s,gpu - A_s,orc| <= (m + p) u sqrt(m'/s)/sqrt(m') sum_i |A_ic| entrywise.
"""
import json
import os

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
DEV = torch.device("cuda", 0)
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_accuracy_levels.json")))


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def status(info):
    return tuple(int(x) for x in info.cpu().tolist())


def nrm2(x):
    return float(np.linalg.norm(x, 2))


@pytest.fixture(scope="module")
def dct_plans(lib):
    ps = {"fp64": lib.rpcholqr_plan_create(0, 1 << 20, 512, 1536),
          "split": lib.rpcholqr_plan_create(0, 1 << 20, 512, 1536, mode=lib.SPLIT64)}
    for p in ps.values():
        lib.rpcholqr_plan_set_smoothing(p, lib.SMOOTH_DCT)
    yield ps
    for p in ps.values():
        p.close()


@pytest.fixture(scope="module")
def smooth_plans(lib):
    ps = {"fp64": lib.rpcholqr_plan_create(0, 1 << 20, 300, 1536),
          "split": lib.rpcholqr_plan_create(0, 1 << 20, 300, 1536, mode=lib.SPLIT64),
          "fp32": lib.rpcholqr_plan_create(0, 1 << 20, 300, 1536, mode=lib.FP32)}
    for p in ps.values():
        lib.rpcholqr_plan_set_smoothing(p, lib.SMOOTH_WHT)
    yield ps
    for p in ps.values():
        p.close()


@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (3, 2, 2), (1000, 7, 21), (2048, 8, 24), (4097, 17, 51),
                                   (70000, 50, 150), ((1 << 20) - 3, 128, 384), (9000, 300, 900)])
def test_smoothed_sample_matches_oracle(lib, oracle_mod, smooth_plans, m, n, s):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, size=(1, n))
    As, info = lib.rpcholqr_smoothed_sample(smooth_plans["fp64"], cu(A), s, 7)
    assert status(info)[0] == 0
    As_o, idx = oracle_mod.smoothed_sample(A, s, 7)
    mp = oracle_mod.smooth_order(m)
    p = int(np.log2(mp))
    bound = (m + p) * EPS / np.sqrt(s) * np.sum(np.abs(A), axis=0)[None, :]
    assert np.all(np.abs(host(As) - As_o) <= bound)


def test_smoothed_sample_nonfinite_anywhere(lib, smooth_plans):
    A = np.ones((5000, 4))
    A[4321, 3] = np.inf
    _, info = lib.rpcholqr_smoothed_sample(smooth_plans["fp64"], cu(A), 12, 1)
    assert status(info)[0] == lib.ERR_NONFINITE


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("m,n,kappa", [(10007, 50, 1e8), (30000, 128, 1e12), (12000, 200, 1e4)])
def test_smoothed_factor_matches_oracle(lib, oracle_mod, smooth_plans, mode, m, n, kappa):
    A = inputs.usv(m, n, kappa, 500 + n)
    s = 3 * n
    Q, R, info = lib.rpcholqr_factor(smooth_plans[mode], cu(A), s, 3)
    assert status(info) == (0, -1)
    o = oracle_mod.rpcholqr(A, s, 3, smoothing=1)
    assert o["status"] == 0
    Qh, Rh = host(Q), host(R)
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    orth = oracle_mod.orth_error(Qh)
    assert orth <= 10 * oracle_mod.orth_error(o["Q"])
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])
    if kappa <= 1e8:
        floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, 3, smoothing=1, variant=1)["Q"])
        assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_coherent_section_5_1_needs_smoothing(lib, oracle_mod, smooth_plans, mode):
    g = GOLD["section_5_1"]
    m, n, kappa = g["workload"]["m"], g["workload"]["n"], g["workload"]["kappa"]
    A = inputs.coherent_randsvd(m, n, kappa, 5)
    plain = lib.rpcholqr_plan_create(0, m, n, 6 * n, mode=lib.SPLIT64 if mode == "split" else lib.FP64)
    try:
        _, _, info = lib.rpcholqr_factor(plain, cu(A), 3 * n, 1)
        assert status(info)[0] == lib.ERR_SINGULAR_SKETCH
    finally:
        plain.close()
    for seed in (1, 2, 3):
        Q, R, info = lib.rpcholqr_factor(smooth_plans[mode], cu(A), 3 * n, seed)
        assert status(info) == (0, -1)
        Qh, Rh = host(Q), host(R)
        o = oracle_mod.rpcholqr(A, 3 * n, seed, smoothing=1)
        # parity: within 10x of the oracle; the paper's levels (residual ~1e-16, orthogonality below
        # 1e-12 at c = 3n) with the same 10x margin for a single trial
        res, orth = oracle_mod.residual(A, Qh, Rh), oracle_mod.orth_error(Qh)
        assert res <= 10 * oracle_mod.residual(A, o["Q"], o["R"]) and res <= 10 * g["residual"]["value"]
        assert orth <= 10 * oracle_mod.orth_error(o["Q"])
        assert orth <= 10 * g["orthogonality_c_3n_all_n"]["value"]
        if mode == "split":
            # kappa(A1) is in the hundreds here: the FP64 second pass is taken
            assert lib.rpcholqr_plan_split_pass2_fp64(smooth_plans[mode])


def test_fp32_with_smoothing_on_coherent_input(lib, smooth_plans):
    m, n = 20000, 64
    A = inputs.coherent_randsvd(m, n, 1e4, 8).astype(np.float32)
    Q, R, info = lib.rpcholqr_factor_f32(smooth_plans["fp32"], torch.from_numpy(A).to(DEV), 3 * n, 2)
    assert status(info) == (0, -1)
    Qd = host(Q).astype(np.float64)
    E = Qd.T @ Qd - np.eye(n)
    assert np.max(np.abs(np.linalg.eigvalsh(E))) <= 1e-5


def test_smoothing_toggles_and_rejects(lib):
    p = lib.rpcholqr_plan_create(0, 4096, 8, 24)
    try:
        with pytest.raises(lib.RpcholqrError):
            lib.rpcholqr_smoothed_sample(p, cu(np.ones((100, 8))), 24, 1)     # smoothing not enabled
        with pytest.raises(lib.RpcholqrError):
            lib.rpcholqr_plan_set_smoothing(p, 7)
        A = cu(inputs.usv(4096, 8, 10.0, 1))
        Q0, R0, _ = lib.rpcholqr_factor(p, A, 24, 5)
        lib.rpcholqr_plan_set_smoothing(p, lib.SMOOTH_WHT)
        Q1, R1, _ = lib.rpcholqr_factor(p, A, 24, 5)
        lib.rpcholqr_plan_set_smoothing(p, lib.SMOOTH_NONE)
        Q2, R2, _ = lib.rpcholqr_factor(p, A, 24, 5)
        assert torch.equal(Q0, Q2) and torch.equal(R0, R2)
        assert not torch.equal(R0, R1)
    finally:
        p.close()


# ---- the cosine transform (Remark r_exp) -------------------------------------------------------------
@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (3, 2, 2), (1000, 7, 21), (2048, 8, 24), (4097, 17, 51),
                                   (70000, 50, 150), ((1 << 20) - 3, 128, 384), (9000, 300, 900)])
def test_dct_sample_matches_oracle(lib, oracle_mod, dct_plans, m, n, s):
    rng = np.random.default_rng(m + 3 * n)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, size=(1, n))
    As, info = lib.rpcholqr_smoothed_sample(dct_plans["fp64"], cu(A), s, 5)
    assert status(info)[0] == 0
    As_o, _ = oracle_mod.smoothed_sample(A, s, 5, kind=oracle_mod.SMOOTH_DCT)
    p = int(np.log2(oracle_mod.smooth_order(m)))
    # the oracle's plain sum (m terms, each with a rounded cosine) and the FFT's p stages of rounded
    # twiddles: entrywise below (m + 8p) u sqrt(2/s) sum_i |A_ic|
    bound = (m + 8 * p + 8) * EPS * np.sqrt(2.0 / s) * np.sum(np.abs(A), axis=0)[None, :]
    assert np.all(np.abs(host(As) - As_o) <= bound)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_dct_factor_matches_oracle(lib, oracle_mod, dct_plans, mode):
    A = inputs.usv(30000, 128, 1e12, 77)
    Q, R, info = lib.rpcholqr_factor(dct_plans[mode], cu(A), 384, 3)
    assert status(info) == (0, -1)
    o = oracle_mod.rpcholqr(A, 384, 3, smoothing=oracle_mod.SMOOTH_DCT)
    Qh, Rh = host(Q), host(R)
    assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
    assert oracle_mod.orth_error(Qh) <= 10 * oracle_mod.orth_error(o["Q"])
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_dct_section_5_1_at_c_2n(lib, oracle_mod, dct_plans, mode):
    # Section 5.1 (Figure fig_ErrorRange3): with the cosine transform even c = 2n = 200 gives a
    # deviation from orthonormality below 1e-12 and residuals near 1e-16 on the coherent inputs
    g = GOLD["section_5_1"]
    m, n, kappa = g["workload"]["m"], g["workload"]["n"], g["workload"]["kappa"]
    A = inputs.coherent_randsvd(m, n, kappa, 5)
    for seed in (1, 2, 3):
        Q, R, info = lib.rpcholqr_factor(dct_plans[mode], cu(A), 2 * n, seed)
        assert status(info) == (0, -1)
        Qh, Rh = host(Q), host(R)
        o = oracle_mod.rpcholqr(A, 2 * n, seed, smoothing=oracle_mod.SMOOTH_DCT)
        orth, res = oracle_mod.orth_error(Qh), oracle_mod.residual(A, Qh, Rh)
        assert orth <= 10 * oracle_mod.orth_error(o["Q"]) and orth <= 10 * g["orthogonality_c_2n"]["value"]
        assert res <= 10 * oracle_mod.residual(A, o["Q"], o["R"]) and res <= 10 * g["residual"]["value"]


@pytest.mark.parametrize("n,s", [(1000, 3000), (2000, 6000)])
def test_dct_sample_wide_matches_oracle(lib, oracle_mod, n, s):
    # the Section 5.1 widths (m = 6000, n = 1000 and 2000): the smoothed sample entrywise against the
    # oracle's within the bound above
    m = 6000
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, size=(1, n))
    plan = lib.rpcholqr_plan_create(0, m, n, s)
    try:
        lib.rpcholqr_plan_set_smoothing(plan, lib.SMOOTH_DCT)
        As, info = lib.rpcholqr_smoothed_sample(plan, cu(A), s, 1)
        assert status(info)[0] == 0
        As_h = host(As)
    finally:
        plan.close()
    As_o, _ = oracle_mod.smoothed_sample(A, s, 1, kind=oracle_mod.SMOOTH_DCT)
    p = int(np.log2(oracle_mod.smooth_order(m)))
    bound = (m + 8 * p + 8) * EPS * np.sqrt(2.0 / s) * np.sum(np.abs(A), axis=0)[None, :]
    assert np.all(np.abs(As_h - As_o) <= bound)
