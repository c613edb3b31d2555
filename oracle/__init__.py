"""FP64 CPU oracle for rpCholesky-QR (Garrison & Ipsen, arXiv 2406.11751) -- TEST INFRASTRUCTURE.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this module only
compiles it, loads it with ctypes and marshals numpy arrays.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library and the CUDA library never calls into it.

Every function follows a step of Algorithm alg_2 ("rpCholesky-QR", Section 4) or of Algorithm
alg_0 ("Basic Cholesky-QR", Section 2.1); the C source states the passage and the reading used.

Error metrics (Section 5):
  * ``orth_error(Q)``    = ||Q^T Q - I||_2 with every entry of Q^T Q a Dot2 compensated sum
                            (Ogita, Rump, Oishi 2005), then the largest |eigenvalue| (numpy
                            ``eigvalsh``, a library step on an n x n symmetric matrix);
  * ``residual(A, Q, R)`` = ||A - Q R||_2 / ||A||_2 with Dot2 residual entries.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NONFINITE", 3: "ERR_SINGULAR_SKETCH", 4: "ERR_NOT_SPD"}
OK, ERR_ARG, ERR_NONFINITE, ERR_SINGULAR_SKETCH, ERR_NOT_SPD = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # RPQ_ORACLE_LIB points the pin tests at a deliberately broken copy (mutation test only)
        lib = ctypes.CDLL(os.environ.get("RPQ_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        U64 = ctypes.c_uint64
        I = ctypes.c_int
        lib.oracle_philox4x64_10.argtypes = [P, P, P]
        lib.oracle_sample_indices.argtypes = [U64, U64, I64, I64, P]
        lib.oracle_gather_scale.argtypes = [P, I64, I64, I64, P, I64, P]
        lib.oracle_householder_r.argtypes = [P, I64, I64, P, I]
        lib.oracle_householder_r.restype = I
        lib.oracle_trsm_rows.argtypes = [P, I64, I64, I64, P, P, I64, I]
        lib.oracle_gram.argtypes = [P, I64, I64, I64, P, I]
        lib.oracle_cholesky_upper.argtypes = [P, I64, P, P, I]
        lib.oracle_cholesky_upper.restype = I
        lib.oracle_triu_mul.argtypes = [P, P, I64, P, I]
        lib.oracle_rpcholqr.argtypes = [P, I64, I64, I64, I64, U64, U64, P, I64, P, P, P, P, P,
                                        P, P, I, I]
        lib.oracle_rpcholqr.restype = I
        lib.oracle_cholqr.argtypes = [P, I64, I64, I64, P, I64, P, P, I]
        lib.oracle_cholqr.restype = I
        lib.oracle_cholqr2.argtypes = [P, I64, I64, I64, P, I64, P, P, I]
        lib.oracle_cholqr2.restype = I
        lib.oracle_orth_matrix.argtypes = [P, I64, I64, I64, P]
        lib.oracle_residual_matrix.argtypes = [P, I64, I64, I64, P, I64, P, P]
        lib.oracle_num_threads.restype = I
        lib.oracle_scholqr3.argtypes = [P, I64, I64, I64, P, I64, P, P, I]
        lib.oracle_scholqr3.restype = I
        lib.oracle_scholqr3_shift.argtypes = [P, I64, I64]
        lib.oracle_scholqr3_shift.restype = ctypes.c_double
        lib.oracle_smooth_order.argtypes = [I64]
        lib.oracle_smooth_order.restype = I64
        lib.oracle_rademacher.argtypes = [U64, U64, I64, P]
        lib.oracle_smooth_rows.argtypes = [P, I64, I64, I64, P, I64, P, I64, P]
        lib.oracle_smoothed_sample.argtypes = [P, I64, I64, I64, I64, U64, U64, I, P, P]
        lib.oracle_smooth_rows_dct.argtypes = [P, I64, I64, I64, P, I64, P, I64, P]
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def philox4x64_10(counter, key) -> np.ndarray:
    """One Philox4x64-10 block: 4 uint64 words for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample_indices(seed: int, m: int, s: int, stream: int = 0) -> np.ndarray:
    idx = np.zeros(s, dtype=np.int64)
    _load().oracle_sample_indices(seed, stream, m, s, _ptr(idx))
    return idx


def gather_scale(A, idx) -> np.ndarray:
    A = _f64(A)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m, n = A.shape
    s = idx.shape[0]
    out = np.zeros((s, n))
    _load().oracle_gather_scale(_ptr(A), m, n, n, _ptr(idx), s, _ptr(out))
    return out


def householder_r(As, variant: int = 0):
    """(R_s, status) of the s x n sample."""
    W = _f64(As).copy()
    s, n = W.shape
    R = np.zeros((n, n))
    st = _load().oracle_householder_r(_ptr(W), s, n, _ptr(R), variant)
    return R, int(st)


def trsm_rows(B, T, variant: int = 0) -> np.ndarray:
    """X = B T^{-1} by row-wise forward substitution (T upper triangular)."""
    B = _f64(B)
    T = _f64(T)
    m, n = B.shape
    X = np.zeros((m, n))
    _load().oracle_trsm_rows(_ptr(B), m, n, n, _ptr(T), _ptr(X), n, variant)
    return X


def gram(X, variant: int = 0) -> np.ndarray:
    X = _f64(X)
    m, n = X.shape
    G = np.zeros((n, n))
    _load().oracle_gram(_ptr(X), m, n, n, _ptr(G), variant)
    return G


def cholesky_upper(G, variant: int = 0):
    """(R, status, pivot) with G = R^T R."""
    G = _f64(G)
    n = G.shape[0]
    R = np.zeros((n, n))
    piv = np.zeros(1, dtype=np.int64)
    st = _load().oracle_cholesky_upper(_ptr(G), n, _ptr(R), _ptr(piv), variant)
    return R, int(st), int(piv[0])


def triu_mul(R2, Rs, variant: int = 0) -> np.ndarray:
    R2 = _f64(R2)
    Rs = _f64(Rs)
    n = R2.shape[0]
    R = np.zeros((n, n))
    _load().oracle_triu_mul(_ptr(R2), _ptr(Rs), n, _ptr(R), variant)
    return R


def rpcholqr(A, s: int, seed: int, stream: int = 0, variant: int = 0, intermediates=False, smoothing: int = 0):
    """rpCholesky-QR of A (m x n).  Returns dict with Q, R, status, pivot (+ idx, Rs, A1, G1, R1).
    smoothing = 1 / 2 samples the Walsh-Hadamard / cosine smoothed F A instead of A (Algorithm alg_2)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    piv = np.zeros(1, dtype=np.int64)
    idx = np.zeros(s, dtype=np.int64)
    Rs = np.zeros((n, n))
    G1 = np.zeros((n, n))
    R1 = np.zeros((n, n))
    A1 = np.zeros((m, n)) if intermediates else None
    st = _load().oracle_rpcholqr(_ptr(A), m, n, n, s, seed, stream, _ptr(Q), n, _ptr(R),
                                 _ptr(idx), _ptr(Rs), _ptr(A1), _ptr(G1), _ptr(R1), _ptr(piv),
                                 variant, smoothing)
    out = {"Q": Q, "R": R, "status": int(st), "pivot": int(piv[0]), "idx": idx, "Rs": Rs,
           "G1": G1, "R1": R1}
    if intermediates:
        out["A1"] = A1
    return out


def smooth_order(m: int) -> int:
    """m' = 2^ceil(log2 m), the order of the Walsh-Hadamard smoothing transform."""
    return int(_load().oracle_smooth_order(m))


def rademacher(seed: int, stream: int, m: int) -> np.ndarray:
    """D_ii in {-1, +1} from bit 63 of the Philox words under key (seed, stream)."""
    d = np.zeros(m)
    _load().oracle_rademacher(seed, stream, m, _ptr(d))
    return d


def smooth_rows(A, d, rows) -> np.ndarray:
    """Rows `rows` of F_T D [A; 0] (F_T the orthogonal Walsh-Hadamard transform of order m')."""
    A = _f64(A)
    m, n = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    d = _f64(d)
    out = np.zeros((rows.shape[0], n))
    _load().oracle_smooth_rows(_ptr(A), m, n, n, _ptr(d), smooth_order(m), _ptr(rows), rows.shape[0],
                               _ptr(out))
    return out


def smooth_rows_dct(A, d, rows) -> np.ndarray:
    """Rows `rows` of F_T D [A; 0] with F_T the orthonormal DCT-II of order m'."""
    A = _f64(A)
    m, n = A.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    d = _f64(d)
    out = np.zeros((rows.shape[0], n))
    _load().oracle_smooth_rows_dct(_ptr(A), m, n, n, _ptr(d), smooth_order(m), _ptr(rows), rows.shape[0],
                                   _ptr(out))
    return out


SMOOTH_WHT, SMOOTH_DCT = 1, 2


def smoothed_sample(A, s: int, seed: int, stream: int = 0, kind: int = SMOOTH_WHT):
    """(A_s, idx): the s-row sample of the smoothed F A (kind 1 Walsh-Hadamard, 2 cosine), scaled by
    sqrt(m'/s)."""
    A = _f64(A)
    m, n = A.shape
    idx = np.zeros(s, dtype=np.int64)
    As = np.zeros((s, n))
    _load().oracle_smoothed_sample(_ptr(A), m, n, n, s, seed, stream, kind, _ptr(idx), _ptr(As))
    return As, idx


def cholqr(A, variant: int = 0):
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    piv = np.zeros(1, dtype=np.int64)
    st = _load().oracle_cholqr(_ptr(A), m, n, n, _ptr(Q), n, _ptr(R), _ptr(piv), variant)
    return {"Q": Q, "R": R, "status": int(st), "pivot": int(piv[0])}


def cholqr2(A, variant: int = 0):
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    piv = np.zeros(1, dtype=np.int64)
    st = _load().oracle_cholqr2(_ptr(A), m, n, n, _ptr(Q), n, _ptr(R), _ptr(piv), variant)
    return {"Q": Q, "R": R, "status": int(st), "pivot": int(piv[0])}


def scholqr3(A, variant: int = 0):
    """Shifted Cholesky-QR3 (the remedy for Cholesky-QR2's breakdown cited in Section 1)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    piv = np.zeros(1, dtype=np.int64)
    st = _load().oracle_scholqr3(_ptr(A), m, n, n, _ptr(Q), n, _ptr(R), _ptr(piv), variant)
    return {"Q": Q, "R": R, "status": int(st), "pivot": int(piv[0])}


def scholqr3_shift(G, m: int) -> float:
    """The shift 11 (m n + n (n + 1)) u trace(G) of shifted Cholesky-QR3 for the n x n Gram matrix G."""
    G = _f64(G)
    return float(_load().oracle_scholqr3_shift(_ptr(G), m, G.shape[0]))


def _sym_norm2(E) -> float:
    w = np.linalg.eigvalsh(0.5 * (E + E.T))
    return float(np.max(np.abs(w)))


def orth_error(Q) -> float:
    """||Q^T Q - I||_2 (Dot2-accurate entries)."""
    Q = _f64(Q)
    m, n = Q.shape
    E = np.zeros((n, n))
    _load().oracle_orth_matrix(_ptr(Q), m, n, n, _ptr(E))
    return _sym_norm2(E)


def residual(A, Q, R) -> float:
    """||A - Q R||_2 / ||A||_2 (Dot2-accurate residual entries)."""
    A = _f64(A)
    Q = _f64(Q)
    R = _f64(R)
    m, n = A.shape
    D = np.zeros((m, n))
    _load().oracle_residual_matrix(_ptr(A), m, n, n, _ptr(Q), n, _ptr(R), _ptr(D))
    nd = np.sqrt(_sym_norm2(D.T @ D))
    na = np.sqrt(_sym_norm2(A.T @ A))
    return float(nd / na)


def orth_error_fast(Q, block: int = 4096) -> float:
    """||Q^T Q - I||_2 with Q^T Q summed over 4096-row blocks (for large m; about eps accurate)."""
    Q = np.asarray(Q, dtype=np.float64)
    m, n = Q.shape
    parts = [Q[i:i + block].T @ Q[i:i + block] for i in range(0, m, block)]
    while len(parts) > 1:
        parts = [parts[i] + parts[i + 1] if i + 1 < len(parts) else parts[i]
                 for i in range(0, len(parts), 2)]
    return _sym_norm2(parts[0] - np.eye(n))
