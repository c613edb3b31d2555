"""GPU tests of the split-precision (SPLIT64) mode: Ozaki-split FP64 products on the BF16 tensor cores.

Reference: FP64 products on the host (numpy) for the product kernels, and the FP64 oracle for the full
factorisation.  Bounds: a split product C = X Y has an absolute error per entry below ~2^-53 times the
power-of-two bounds of its row of X and column of Y (times a small constant for the dropped slice pairs
and the truncation); the full factorisation must reach ||Q^T Q - I|| <= 1e-13 (the benchmark's gate)
and match the oracle's R to 1e-12 and its orthogonality and residual within 10x.
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


def pow2_bound(v, axis):
    mx = np.max(np.abs(v), axis=axis)
    return np.where(mx > 0, 2.0 ** (np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 1), 0.0)


@pytest.fixture(scope="module")
def splan(lib):
    p = lib.rpcholqr_plan_create(0, 1 << 20, 128, 1536, mode=lib.SPLIT64)
    yield p
    p.close()


@pytest.mark.parametrize("m,K,N", [(128, 16, 64), (1000, 128, 128), (4099, 50, 50), (300, 64, 100),
                                   (129, 7, 1), (20000, 128, 64)])
def test_ozaki_gemm_matches_fp64(lib, splan, m, K, N):
    rng = np.random.default_rng(m + K + N)
    X = rng.standard_normal((m, K)) * (10.0 ** rng.uniform(-6, 6, size=(m, 1)))
    Y = np.triu(rng.standard_normal((K, N)) * (10.0 ** rng.uniform(-3, 3, size=(1, N))))
    C, info = lib.rpcholqr_ozaki_gemm(splan, cu(X), cu(Y))
    assert int(info[0]) == 0
    ref = X @ Y
    scale = pow2_bound(X, 1)[:, None] * pow2_bound(Y, 0)[None, :]
    err = np.abs(host(C) - ref)
    assert np.max(err / np.maximum(scale, 1e-300)) <= 8 * K * EPS


# C = B - X Y: K <= 32 runs the first pass's update kernel (staged rows, B/C tiles in shared memory),
# larger K the windowed product in subtract form.  Views with row strides wider than the matrix (odd
# ones: rows not 16-byte aligned), ragged m, K and N, many row blocks per CTA, and C == B in place.
@pytest.mark.parametrize("m,K,N,layout", [(128, 16, 48, "plain"), (1000, 16, 32, "plain"), (4099, 32, 96, "plain"),
                                          (70001, 16, 48, "view"), (300, 9, 37, "odd"), (257, 32, 128, "inplace"),
                                          (262147, 16, 16, "inplace"), (5000, 64, 64, "view"), (129, 1, 1, "plain")])
def test_ozaki_update_matches_fp64(lib, splan, m, K, N, layout):
    rng = np.random.default_rng(7 * m + K + N)
    X = rng.standard_normal((m, K)) * (10.0 ** rng.uniform(-6, 6, size=(m, 1)))
    Y = np.triu(rng.standard_normal((K, N)) * (10.0 ** rng.uniform(-3, 3, size=(1, N))), 1 - K)
    B = rng.standard_normal((m, N)) * (10.0 ** rng.uniform(-4, 4, size=(m, 1)))
    if layout == "plain" or layout == "inplace":
        Xd, Bd = cu(X), cu(B)
    else:
        # columns of wider matrices: row strides K + 16 / N + 8, or odd ones (unaligned rows)
        wx, wb = (K + 16, N + 8) if layout == "view" else (K + 5, N + 3)
        Xw = torch.zeros((m, wx), dtype=torch.float64, device=DEV)
        Bw = torch.zeros((m, wb), dtype=torch.float64, device=DEV)
        Xd, Bd = Xw[:, 3:3 + K], Bw[:, 1:1 + N]
        Xd.copy_(cu(X))
        Bd.copy_(cu(B))
    C, info = lib.rpcholqr_ozaki_update(splan, Xd, cu(Y), Bd, C=Bd if layout == "inplace" else None)
    assert int(info[0]) == 0
    ref = B - X @ Y
    scale = pow2_bound(X, 1)[:, None] * pow2_bound(Y, 0)[None, :]
    err = np.abs(host(C) - ref)
    assert np.all(err <= 8 * K * EPS * scale + 2 * EPS * np.abs(ref))


def test_ozaki_gemm_exact_on_small_integers(lib, splan):
    # integer inputs with few bits: every slice product and sum is exact, so is the result
    rng = np.random.default_rng(3)
    X = rng.integers(-1000, 1000, size=(777, 96)).astype(np.float64)
    Y = rng.integers(-1000, 1000, size=(96, 80)).astype(np.float64)
    C, info = lib.rpcholqr_ozaki_gemm(splan, cu(X), cu(Y))
    assert int(info[0]) == 0
    assert np.array_equal(host(C), X @ Y)


@pytest.mark.parametrize("m,n", [(128, 16), (10007, 50), (70001, 128), (5000, 100), (300, 1)])
def test_ozaki_gram_matches_fp64(lib, oracle_mod, splan, m, n):
    A = inputs.usv(m, n, 1e3, m + n)
    rs = oracle_mod.rpcholqr(A, 3 * n if 3 * n <= m else m, 1, intermediates=True)
    A1 = rs["A1"]                                   # a well-conditioned input like the method's
    G, info = lib.rpcholqr_ozaki_gram(splan, cu(A1))
    assert int(info[0]) == 0
    ref = oracle_mod.gram(A1)
    Gh = host(G)
    assert np.array_equal(Gh, Gh.T)
    assert np.linalg.norm(Gh - ref, 2) <= 4e-15 * np.linalg.norm(ref, 2)


@pytest.mark.parametrize("m,n,kappa", [(10007, 50, 1e8), (20000, 128, 1e4), (50000, 100, 1e12),
                                       (30011, 64, 1e16), (4096, 7, 1.0), (70001, 128, 1e8)])
def test_split_factor_matches_oracle(lib, oracle_mod, splan, m, n, kappa):
    A = inputs.usv(m, n, kappa, 700 + n)
    s = 3 * n
    Q, R, info = lib.rpcholqr_factor(splan, cu(A), s, 5)
    assert info.cpu().tolist() == [0, -1]
    o = oracle_mod.rpcholqr(A, s, 5)
    Qh, Rh = host(Q), host(R)
    assert np.linalg.norm(Rh - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
    orth = oracle_mod.orth_error(Qh)
    assert orth <= 1e-13 and orth <= 10 * oracle_mod.orth_error(o["Q"])
    assert oracle_mod.residual(A, Qh, Rh) <= 10 * oracle_mod.residual(A, o["Q"], o["R"])
    if kappa <= 1e8:
        floor = np.linalg.norm(o["Q"] - oracle_mod.rpcholqr(A, s, 5, variant=1)["Q"], 2)
        assert np.linalg.norm(Qh - o["Q"], 2) <= max(1e-10, 10 * floor)
    # incoherent A: A1 is well conditioned and the tensor-core second pass is kept
    assert not lib.rpcholqr_plan_split_pass2_fp64(splan)


def test_split_factor_nonfinite(lib, oracle_mod, splan):
    A = inputs.usv(9000, 100, 10.0, 5)
    idx = set(oracle_mod.sample_indices(3, 9000, 300).tolist())
    A[next(i for i in range(9000) if i not in idx), 77] = np.nan
    _, _, info = lib.rpcholqr_factor(splan, cu(A), 300, 3)
    assert int(info[0]) == lib.ERR_NONFINITE


def test_split_factor_deterministic(lib, splan):
    A = cu(inputs.usv(40000, 128, 1e10, 8))
    Q1, R1, _ = lib.rpcholqr_factor(splan, A, 384, 11)
    Q2, R2, _ = lib.rpcholqr_factor(splan, A, 384, 11)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


@pytest.mark.parametrize("m,n,s,kappa", [(70001, 128, 384, 1e8), (20011, 50, 150, 1e12), (600, 20, 60, 1e4)])
def test_split_factor_host_matches_device(lib, splan, m, n, s, kappa):
    # the host-buffer call overlaps its copies with the work (row blocks of A copied while earlier ones
    # are solved, Q copied back block by block) but takes the same steps: results identical to the
    # device-buffer call, on two calls in a row
    A = inputs.usv(m, n, kappa, m % 97)
    Qd, Rd, infod = lib.rpcholqr_factor(splan, cu(A), s, 21)
    assert int(infod[0]) == 0
    Ah = torch.from_numpy(A).pin_memory()
    for _ in range(2):
        Qh, Rh, st, piv = lib.rpcholqr_factor_host(splan, Ah, s, 21)
        assert (st, piv) == (0, -1)
        assert np.array_equal(Qh.numpy(), host(Qd)) and np.array_equal(Rh.numpy(), host(Rd))


def test_split_factor_host_nonfinite(lib, oracle_mod, splan):
    # a NaN outside the sample is caught by pass 1, one inside it by the sample (gathered on the host)
    m, n, s = 9000, 100, 300
    idx = oracle_mod.sample_indices(3, m, s).tolist()
    for row in (next(i for i in range(m) if i not in set(idx)), idx[7]):
        A = inputs.usv(m, n, 10.0, 5)
        A[row, 77] = np.nan
        _, _, st, _ = lib.rpcholqr_factor_host(splan, torch.from_numpy(A).pin_memory(), s, 3)
        assert st == lib.ERR_NONFINITE
