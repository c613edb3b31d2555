"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks one oracle step against something other than the oracle itself: an independent
implementation (numpy's Philox4x64-10, LAPACK through numpy/scipy), a closed form, an invariant,
the paper's stated accuracy levels (tests/golden/), or a lemma of the paper.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.linalg

import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- Philox4x64-10 / sampling (the paper's randi, Remark r_exp; our published-generator reading) ---
@pytest.mark.parametrize("key", [(0, 0), (12345, 0), (7, 3), (2**64 - 1, 2**63 + 5)])
def test_philox_matches_numpy(oracle_mod, key):
    # numpy.random.Philox is an independent Philox4x64-10; its n-th block is counter n+1 of ours.
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.zeros(4, dtype=np.uint64))
    raw = bg.random_raw(4 * 6)
    for blk in range(6):
        ours = oracle_mod.philox4x64_10([blk + 1, 0, 0, 0], key)
        assert np.array_equal(ours, raw[4 * blk:4 * blk + 4])


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox4x64_10([5, 6, 7, 8], (9, 10))
    for w in range(4):
        c = [5, 6, 7, 8]
        c[w] += 1
        assert not np.array_equal(oracle_mod.philox4x64_10(c, (9, 10)), base)


@pytest.mark.parametrize("m,s,seed", [(10, 37, 1), (10000, 150, 2), (2**40 + 3, 64, 3), (1, 5, 4)])
def test_sample_indices_from_philox_words(oracle_mod, m, s, seed):
    idx = oracle_mod.sample_indices(seed, m, s)
    # numpy increments its 256-bit counter before each block: all-ones wraps to our block 0
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                          counter=np.full(4, 2**64 - 1, dtype=np.uint64))
    words = bg.random_raw(((s + 3) // 4) * 4)
    expect = [(int(words[j]) * m) >> 64 for j in range(s)]
    assert idx.tolist() == expect
    assert idx.min() >= 0 and idx.max() < m


def test_sample_indices_uniform(oracle_mod):
    m, s = 16, 64000
    idx = oracle_mod.sample_indices(99, m, s)
    counts = np.bincount(idx, minlength=m)
    chi2 = float(((counts - s / m) ** 2 / (s / m)).sum())
    assert chi2 < 50.0   # 15 dof: P(chi2 > 50) ~ 1e-5


def test_gather_scale(oracle_mod):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 4))
    idx = np.array([3, 3, 49, 0, 17])
    As = oracle_mod.gather_scale(A, idx)
    assert np.array_equal(As, np.sqrt(50 / 5) * A[idx])


# ---- Householder QR of the sample (step 'factor A_s = Q_s R_s') -----------------------------------
@pytest.mark.parametrize("s,n", [(12, 5), (30, 30), (7, 1), (64, 9)])
def test_householder_matches_lapack(oracle_mod, s, n):
    rng = np.random.default_rng(s * 100 + n)
    As = rng.standard_normal((s, n)) * np.logspace(0, -6, n)[None, :]
    R, st = oracle_mod.householder_r(As)
    assert st == 0
    r_np = np.linalg.qr(As, mode="r")
    r_np = r_np * np.sign(np.diag(r_np))[:, None]
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.linalg.norm(R - r_np) <= 50 * EPS * np.linalg.norm(r_np)
    assert np.linalg.norm(R.T @ R - As.T @ As) <= 50 * EPS * np.linalg.norm(As) ** 2


def test_householder_closed_form(oracle_mod):
    As = np.array([[3.0, 0.0], [4.0, 0.0], [0.0, 5.0]])
    R, st = oracle_mod.householder_r(As)
    assert st == 0
    assert np.allclose(R, [[5.0, 0.0], [0.0, 5.0]], rtol=0, atol=4 * EPS * 5)


def test_householder_zero_column_is_singular(oracle_mod):
    As = np.array([[1.0, 0.0, 2.0], [2.0, 0.0, 1.0], [0.5, 0.0, 3.0], [1.0, 0.0, 1.0]])
    _, st = oracle_mod.householder_r(As)
    assert st == oracle_mod.ERR_SINGULAR_SKETCH


# ---- row-wise triangular solve, Gram, Cholesky, triangular product --------------------------------
def test_trsm_rows_matches_scipy(oracle_mod):
    rng = np.random.default_rng(5)
    T = np.triu(rng.standard_normal((9, 9))) + 4 * np.eye(9)
    B = rng.standard_normal((40, 9))
    X = oracle_mod.trsm_rows(B, T)
    ref = scipy.linalg.solve_triangular(T.T, B.T, lower=True).T
    assert np.allclose(X, ref, rtol=1e-13, atol=1e-14)
    assert np.allclose(X @ T, B, rtol=0, atol=1e-13)


def test_gram_matches_numpy(oracle_mod):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((9000, 7))   # spans three 4096-row blocks
    G = oracle_mod.gram(X)
    assert np.allclose(G, X.T @ X, rtol=1e-13, atol=1e-10)
    assert np.array_equal(G, G.T)


def test_cholesky_matches_numpy(oracle_mod):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((50, 8))
    G = X.T @ X
    R, st, piv = oracle_mod.cholesky_upper(G)
    assert st == 0 and piv == -1
    assert np.allclose(R, np.linalg.cholesky(G).T, rtol=1e-13, atol=1e-13)


def test_cholesky_not_spd_reports_pivot(oracle_mod):
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    _, st, piv = oracle_mod.cholesky_upper(G)
    assert st == oracle_mod.ERR_NOT_SPD and piv == 2
    G = np.eye(3)
    G[1, 1] = np.nan
    _, st, piv = oracle_mod.cholesky_upper(G)
    assert st == oracle_mod.ERR_NOT_SPD and piv == 1


def test_triu_mul_matches_numpy(oracle_mod):
    rng = np.random.default_rng(8)
    a = np.triu(rng.standard_normal((6, 6)))
    b = np.triu(rng.standard_normal((6, 6)))
    assert np.allclose(oracle_mod.triu_mul(a, b), a @ b, rtol=1e-14, atol=1e-14)


# ---- whole pipeline --------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,kappa", [(200, 6, 1e3), (500, 17, 1e6), (64, 8, 10.0)])
def test_rpcholqr_equals_unique_qr(oracle_mod, m, n, kappa):
    # Lemma l_r1r2 / Remark r_precond: with diag(R) > 0 the thin QR is unique and rpCholesky-QR
    # reaches it for any nonsingular R_s; compare with LAPACK's Householder QR, sign-normalised.
    A = inputs.usv(m, n, kappa, 11)
    o = oracle_mod.rpcholqr(A, 3 * n, 5)
    assert o["status"] == 0
    q, r = np.linalg.qr(A)
    d = np.sign(np.diag(r))
    q, r = q * d[None, :], r * d[:, None]
    assert np.linalg.norm(o["R"] - r, 2) <= 1e-13 * np.linalg.norm(r, 2)
    assert np.linalg.norm(o["Q"] - q, 2) <= 1e-14 * kappa
    assert np.all(np.diag(o["R"]) > 0)


def test_n1_closed_form(oracle_mod):
    rng = np.random.default_rng(12)
    a = rng.standard_normal((300, 1))
    o = oracle_mod.rpcholqr(a, 3, 1)
    nrm = np.sqrt(np.sum(a * a))
    assert o["status"] == 0
    assert abs(o["R"][0, 0] - nrm) <= 8 * EPS * nrm
    assert np.max(np.abs(o["Q"] - a / nrm)) <= 8 * EPS * np.max(np.abs(a / nrm))


def test_orthonormal_input_gives_identity(oracle_mod):
    u, _, _ = inputs.usv_factors(2000, 20, 1.0, 3)
    o = oracle_mod.rpcholqr(u, 60, 9)
    assert o["status"] == 0
    assert np.linalg.norm(o["R"] - np.eye(20), 2) <= 1e-14
    assert np.linalg.norm(o["Q"] - u, 2) <= 1e-14


def test_scale_equivariance_bit_exact(oracle_mod):
    A = inputs.usv(700, 9, 1e5, 13)
    o = oracle_mod.rpcholqr(A, 27, 3)
    # global power-of-two scale
    o2 = oracle_mod.rpcholqr(A * 2.0 ** 7, 27, 3)
    assert np.array_equal(o2["Q"], o["Q"])
    assert np.array_equal(o2["R"], o["R"] * 2.0 ** 7)
    # column scaling by powers of two: Q unchanged, R -> R D (every step is column-equivariant)
    d = 2.0 ** np.array([3, -2, 0, 5, -7, 1, 2, -1, 4])
    o3 = oracle_mod.rpcholqr(A * d[None, :], 27, 3)
    assert np.array_equal(o3["Q"], o["Q"])
    assert np.array_equal(o3["R"], o["R"] * d[None, :])


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e10])
def test_lemma_l31_singular_values_of_A1(oracle_mod, kappa):
    # Lemma l_31: sigma_i(S F Q) = 1 / sigma_{n-i+1}(A_1); here F = I, S carries sqrt(m/s) and the
    # orthonormal factor of A is U W (W orthogonal), so the singular values are those of
    # sqrt(m/s) U[idx, :].  kappa(R_1) = kappa(A_1) because G_1 = A_1^T A_1 = R_1^T R_1.
    m, n, s = 3000, 12, 36
    A, (u, _, _) = inputs.usv(m, n, kappa, 21, return_factors=True)
    o = oracle_mod.rpcholqr(A, s, 4, intermediates=True)
    assert o["status"] == 0
    sv_sample = np.linalg.svd(np.sqrt(m / s) * u[o["idx"]], compute_uv=False)
    sv_a1 = np.linalg.svd(o["A1"], compute_uv=False)
    assert np.allclose(np.sort(1.0 / sv_sample), np.sort(sv_a1), rtol=1e-9 * max(1.0, kappa / 1e4))
    sv_r1 = np.linalg.svd(o["R1"], compute_uv=False)
    assert np.allclose(np.sort(sv_r1), np.sort(sv_a1), rtol=1e-12)


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12, 1e15, 1e16])
def test_orthogonality_tracks_kappa_A1_not_kappa_A_squared(oracle_mod, kappa):
    # Section 5.2, Eq. e_ex1: ||Q^T Q - I|| ~ 4 eps kappa(A_1); first-order bound of Corollary
    # c_perturb2 is ~ 4 eps kappa(A_1)^2; the residual stays at machine precision (Section 5.1).
    m, n, s = 6000, 40, 120
    A = inputs.usv(m, n, kappa, 31)
    o = oracle_mod.rpcholqr(A, s, 6)
    assert o["status"] == 0
    k1 = np.linalg.cond(o["R1"])
    orth = oracle_mod.orth_error(o["Q"])
    res = oracle_mod.residual(A, o["Q"], o["R"])
    assert orth <= 20 * EPS * k1
    assert orth <= 1e-13 and orth < EPS * kappa ** 2
    assert res <= 1e-15
    # theorem-level sanity: Theorem t_perturb2 bound with eps_i = n u
    g1 = 4 * n * EPS
    g2 = 3 * n * EPS
    assert orth <= k1 ** 2 * g1 / (1 - k1 ** 2 * g2)


def test_cholqr2_breaks_down_where_rpcholqr_does_not(oracle_mod):
    A = inputs.usv(6000, 40, 1e16, 32)
    assert oracle_mod.cholqr2(A)["status"] == oracle_mod.ERR_NOT_SPD
    o = oracle_mod.rpcholqr(A, 120, 2)
    assert o["status"] == 0
    assert oracle_mod.orth_error(o["Q"]) <= 1e-13


def test_paper_section53_accuracy_levels(oracle_mod):
    # tests/golden/paper_accuracy_levels.json: Haar Q_A times randsvd(n, 1e7), c = 3n, 10 trials.
    gold = json.load(open(os.path.join(GOLDEN, "paper_accuracy_levels.json")))
    wl = gold["workload"]
    m, n = wl["m"], 60
    A = inputs.usv(m, n, wl["kappa"], 41)
    c2 = oracle_mod.cholqr2(A)
    assert c2["status"] == 0
    c2_orth = oracle_mod.orth_error(c2["Q"])
    for trial in range(wl["trials"]):
        o = oracle_mod.rpcholqr(A, wl["c_over_n"] * n, 100 + trial)
        assert o["status"] == 0
        res = oracle_mod.residual(A, o["Q"], o["R"])
        orth = oracle_mod.orth_error(o["Q"])
        assert gold["rpcholqr"]["residual"]["value"] <= res * 10 and res < 1e-15   # ~1e-16
        assert orth < 2e-14                                                             # ~1e-15
        assert orth < 20 * c2_orth + 1e-14                                              # same magnitude


# ---- error paths -----------------------------------------------------------------------------------
def test_nonfinite_input(oracle_mod):
    A = inputs.usv(500, 5, 10.0, 1)
    A[123, 2] = np.nan
    o = oracle_mod.rpcholqr(A, 15, 1)
    assert o["status"] == oracle_mod.ERR_NONFINITE


def test_coherent_input_gives_singular_sketch(oracle_mod):
    # [D; 0] (the worst-coherence shape of Eq. e_ErrorRange): without smoothing a uniform sample of
    # 3n rows out of m >> n almost surely misses a row of D, leaving a zero column in A_s.
    A = inputs.coherent_diag(5000, 10, 1)
    o = oracle_mod.rpcholqr(A, 30, 1)
    missed = set(range(10)) - set(o["idx"].tolist())
    assert missed and o["status"] == oracle_mod.ERR_SINGULAR_SKETCH


def test_bad_arguments(oracle_mod):
    A = np.ones((10, 4))
    assert oracle_mod.rpcholqr(A, 3, 1)["status"] == oracle_mod.ERR_ARG    # s < n
    assert oracle_mod.rpcholqr(A, 11, 1)["status"] == oracle_mod.ERR_ARG   # s > m


# ---- metrics and determinism -----------------------------------------------------------------------
def test_metrics_closed_forms(oracle_mod):
    q = np.zeros((100, 3))
    q[[5, 50, 99], [0, 1, 2]] = 1.0
    assert oracle_mod.orth_error(q) == 0.0
    # (1 + 2^-33)^2 - 1 = 2^-32 + 2^-66 exactly; Dot2 must resolve the 2^-66 term
    assert oracle_mod.orth_error(q * (1 + 2.0 ** -33)) == 2.0 ** -32 + 2.0 ** -66
    A = inputs.usv(300, 5, 100.0, 2)
    q, r = np.linalg.qr(A)
    assert oracle_mod.residual(A, q, r) < 1e-15


def test_result_independent_of_thread_count(oracle_mod):
    code = ("import sys, hashlib; sys.path.insert(0, %r); import oracle, inputs;"
            "o = oracle.rpcholqr(inputs.usv(9000, 16, 1e6, 5), 48, 3);"
            "print(hashlib.sha256(o['Q'].tobytes() + o['R'].tobytes()).hexdigest())"
            % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    outs = []
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                                   text=True, check=True).stdout.strip())
    assert outs[0] == outs[1]


def test_two_roundings_agree_in_R_and_to_eps_kappa_in_Q(oracle_mod):
    # The parity floor: two valid summation orders give R equal to ~eps (normwise) at every kappa,
    # Q equal to ~eps kappa(A) (the QR factor's own conditioning).
    for kappa in (1e2, 1e8):
        A = inputs.usv(4000, 24, kappa, 51)
        a = oracle_mod.rpcholqr(A, 72, 8)
        b = oracle_mod.rpcholqr(A, 72, 8, variant=1)
        assert np.linalg.norm(a["R"] - b["R"], 2) <= 1e-14 * np.linalg.norm(a["R"], 2)
        assert np.linalg.norm(a["Q"] - b["Q"], 2) <= 1e3 * EPS * kappa


# ---- shifted Cholesky-QR3 (cited in Section 1 as the remedy for Cholesky-QR2's breakdown) ------------
def test_scholqr3_shift_closed_form(oracle_mod):
    G = np.diag([4.0, 9.0, 1.0])
    assert oracle_mod.scholqr3_shift(G, 10) == 11.0 * (10 * 3 + 3 * 4) * 2.0 ** -53 * 14.0


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12])
def test_scholqr3_succeeds_where_cholqr2_breaks_down(oracle_mod, kappa):
    m, n = 3000, 40
    A = inputs.usv(m, n, kappa, 51)
    o3 = oracle_mod.scholqr3(A)
    assert o3["status"] == 0
    # LAPACK QR fixes the answer up to column signs; sCholQR3's R has a positive diagonal
    q, r = np.linalg.qr(A)
    sgn = np.sign(np.diag(r))
    assert np.all(np.diag(o3["R"]) > 0)
    assert oracle_mod.orth_error(o3["Q"]) <= 1e-14
    assert oracle_mod.residual(A, o3["Q"], o3["R"]) <= 1e-15
    if kappa <= 1e8:
        assert np.linalg.norm(o3["R"] - sgn[:, None] * r, 2) <= 1e-12 * kappa * np.linalg.norm(r, 2)
    if kappa >= 1e12:
        assert oracle_mod.cholqr2(A)["status"] == oracle_mod.ERR_NOT_SPD


def test_scholqr3_range_ends_where_rpcholqr_still_works(oracle_mod):
    # the shifted first stage leaves kappa(Q_1) ~ sqrt(sigma) kappa(A) (sigma the shift), which
    # Cholesky-QR2 needs below ~u^-1/2: at kappa(A) = 1e15 the method breaks down, while
    # rpCholesky-QR handles numerically singular A (Section 5.1)
    A = inputs.usv(3000, 40, 1e15, 51)
    G = oracle_mod.gram(A)
    sigma = oracle_mod.scholqr3_shift(G, 3000)
    assert 1e-11 < sigma < 1e-9
    assert oracle_mod.scholqr3(A)["status"] == oracle_mod.ERR_NOT_SPD
    o = oracle_mod.rpcholqr(A, 120, 1)
    assert o["status"] == 0 and oracle_mod.orth_error(o["Q"]) <= 1e-13
