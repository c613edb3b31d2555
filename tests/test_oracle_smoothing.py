"""Pins of the oracle's smoothing F = F_T D (Algorithm alg_2 line 2; the Blendenpik remark of
Section 4; Remark r_exp) against things other than itself: numpy's Philox for the Rademacher signs,
scipy's Hadamard matrix for F_T, orthogonality (norm preservation), an independent fast Walsh-Hadamard
transform, the zero-padding reading, and the accuracy levels Section 5.1 states for the maximally
coherent matrices of Eq. e_ErrorRange."""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_accuracy_levels.json")))


@pytest.mark.parametrize("seed,stream,m", [(1, 1, 37), (2**63 + 5, 1, 400), (7, 9, 4)])
def test_rademacher_from_philox_bit63(oracle_mod, seed, stream, m):
    # numpy increments its 256-bit counter before each block: all-ones wraps to our block 0
    bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64),
                          counter=np.full(4, np.iinfo(np.uint64).max, dtype=np.uint64))
    words = bg.random_raw((m + 3) // 4 * 4).astype(np.uint64)
    ref = np.where((words[:m] >> np.uint64(63)) != 0, -1.0, 1.0)
    assert np.array_equal(oracle_mod.rademacher(seed, stream, m), ref)


def test_rademacher_is_balanced(oracle_mod):
    d = oracle_mod.rademacher(3, 1, 100000)
    assert set(np.unique(d)) == {-1.0, 1.0}
    assert abs(d.mean()) < 0.02


@pytest.mark.parametrize("mp", [1, 2, 8, 64])
def test_transform_is_sylvester_hadamard(oracle_mod, mp):
    d = oracle_mod.rademacher(5, 1, mp)
    F = oracle_mod.smooth_rows(np.eye(mp), d, np.arange(mp))
    assert np.array_equal(F, scipy.linalg.hadamard(mp) * d[None, :] / np.sqrt(mp))


def test_order_is_next_power_of_two(oracle_mod):
    for m, mp in [(1, 1), (2, 2), (3, 4), (300, 512), (512, 512), (513, 1024), (6000, 8192)]:
        assert oracle_mod.smooth_order(m) == mp


def test_smoothing_is_orthogonal_and_pads_with_zeros(oracle_mod):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((300, 7))
    d = oracle_mod.rademacher(11, 1, 300)
    FA = oracle_mod.smooth_rows(A, d, np.arange(512))
    G = A.T @ A
    assert np.linalg.norm(FA.T @ FA - G, 2) <= 1e-13 * np.linalg.norm(G, 2)
    # [A; 0] with 212 explicit zero rows (any signs there) gives the same rows bit for bit
    Ap = np.vstack([A, np.zeros((212, 7))])
    dp = np.concatenate([d, oracle_mod.rademacher(99, 1, 212)])
    assert np.array_equal(oracle_mod.smooth_rows(Ap, dp, np.arange(512)), FA)


def _fwht(X):
    X = X.copy()
    h = 1
    while h < X.shape[0]:
        for i in range(0, X.shape[0], 2 * h):
            a = X[i:i + h].copy()
            b = X[i + h:i + 2 * h].copy()
            X[i:i + h] = a + b
            X[i + h:i + 2 * h] = a - b
        h *= 2
    return X


def test_direct_rows_match_fast_transform(oracle_mod):
    rng = np.random.default_rng(1)
    m, n = 1000, 5
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1))
    d = oracle_mod.rademacher(4, 1, m)
    mp = 1024
    X = np.zeros((mp, n))
    X[:m] = d[:, None] * A
    ref = _fwht(X) / np.sqrt(mp)
    rows = np.array([0, 1, 2, 511, 512, 1000, 1023, 77])
    got = oracle_mod.smooth_rows(A, d, rows)
    assert np.max(np.abs(got - ref[rows])) <= 1e-12 * np.max(np.abs(A))


def test_smoothed_sample_is_scaled_rows_of_FA(oracle_mod):
    rng = np.random.default_rng(2)
    m, n, s, seed = 700, 6, 18, 21
    A = rng.standard_normal((m, n))
    As, idx = oracle_mod.smoothed_sample(A, s, seed)
    mp = 1024
    assert np.array_equal(idx, oracle_mod.sample_indices(seed, mp, s))
    rows = oracle_mod.smooth_rows(A, oracle_mod.rademacher(seed, 1, m), idx)
    assert np.array_equal(As, rows * np.sqrt(mp / s))


def test_coherent_inputs_need_smoothing_section_5_1(oracle_mod):
    g = GOLD["section_5_1"]
    m, n, kappa = g["workload"]["m"], g["workload"]["n"], g["workload"]["kappa"]
    A = inputs.coherent_randsvd(m, n, kappa, 5)
    # without F the sample almost surely misses one of the n nonzero rows: R_s is singular
    assert oracle_mod.rpcholqr(A, 3 * n, 1)["status"] == oracle_mod.ERR_SINGULAR_SKETCH
    for seed in (1, 2, 3):
        o = oracle_mod.rpcholqr(A, 3 * n, seed, smoothing=1, intermediates=True)
        assert o["status"] == 0
        assert oracle_mod.residual(A, o["Q"], o["R"]) <= 10 * g["residual"]["value"]
        assert oracle_mod.orth_error(o["Q"]) <= g["orthogonality_c_3n_all_n"]["value"]
    # c = 6n: kappa(A_1) below 10 and orthogonality about 1e-15
    o = oracle_mod.rpcholqr(A, 6 * n, 4, smoothing=1, intermediates=True)
    sv = np.linalg.svd(o["A1"], compute_uv=False)
    assert sv[0] / sv[-1] < g["kappa_A1_c_ge_6n"]["value"]
    assert oracle_mod.orth_error(o["Q"]) <= 10 * g["orthogonality_c_ge_6n"]["value"]


def test_smoothing_reports_nonfinite_anywhere(oracle_mod):
    A = inputs.usv(500, 4, 10.0, 1)
    A[123, 2] = np.nan
    assert oracle_mod.rpcholqr(A, 12, 1, smoothing=1)["status"] == oracle_mod.ERR_NONFINITE


# ---- the cosine transform (Remark r_exp uses MATLAB's dct) ----------------------------------------------
@pytest.mark.parametrize("mp", [1, 2, 8, 64, 1024])
def test_dct_rows_are_scipy_orthonormal_dct(oracle_mod, mp):
    import scipy.fft
    d = oracle_mod.rademacher(6, 1, mp)
    F = oracle_mod.smooth_rows_dct(np.eye(mp), d, np.arange(mp))
    ref = scipy.fft.dct(np.diag(d), type=2, norm="ortho", axis=0)
    assert np.max(np.abs(F - ref)) <= 4 * np.finfo(float).eps


def test_dct_is_orthogonal_and_pads_with_zeros(oracle_mod):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((300, 6))
    d = oracle_mod.rademacher(8, 1, 300)
    FA = oracle_mod.smooth_rows_dct(A, d, np.arange(512))
    G = A.T @ A
    assert np.linalg.norm(FA.T @ FA - G, 2) <= 1e-13 * np.linalg.norm(G, 2)
    Ap = np.vstack([A, np.zeros((212, 6))])
    dp = np.concatenate([d, oracle_mod.rademacher(5, 1, 212)])
    assert np.array_equal(oracle_mod.smooth_rows_dct(Ap, dp, np.arange(512)), FA)


def test_dct_smoothed_sample(oracle_mod):
    rng = np.random.default_rng(9)
    m, n, s, seed = 700, 5, 15, 4
    A = rng.standard_normal((m, n))
    As, idx = oracle_mod.smoothed_sample(A, s, seed, kind=oracle_mod.SMOOTH_DCT)
    assert np.array_equal(idx, oracle_mod.sample_indices(seed, 1024, s))
    rows = oracle_mod.smooth_rows_dct(A, oracle_mod.rademacher(seed, 1, m), idx)
    assert np.array_equal(As, rows * np.sqrt(1024 / s))


def test_dct_smoothing_section_5_1_at_c_2n(oracle_mod):
    # with the cosine transform even c = 2n gives deviation from orthonormality below 1e-12
    # (Section 5.1, Figure fig_ErrorRange3); the Walsh-Hadamard rows restricted to the first n
    # columns repeat with period 2^ceil(log2 n), which c = 2n draws do not reliably cover
    g = GOLD["section_5_1"]
    m, n, kappa = g["workload"]["m"], g["workload"]["n"], g["workload"]["kappa"]
    A = inputs.coherent_randsvd(m, n, kappa, 5)
    for seed in (1, 2, 3):
        o = oracle_mod.rpcholqr(A, 2 * n, seed, smoothing=oracle_mod.SMOOTH_DCT)
        assert o["status"] == 0
        assert oracle_mod.orth_error(o["Q"]) <= g["orthogonality_c_2n"]["value"]
        assert oracle_mod.residual(A, o["Q"], o["R"]) <= 10 * g["residual"]["value"]
