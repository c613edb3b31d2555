"""Seeded synthetic inputs for rpCholesky-QR (Garrison & Ipsen, arXiv 2406.11751).

This module holds no arithmetic of the method itself: it only draws test matrices. Both the
FP64 oracle (``oracle/``) and the CUDA path (via ``bench.py`` and the tests) take their inputs
from here, so the two sides see identical bits.

Recipes (all FP64, row-major m x n):

* ``usv(m, n, kappa, seed)`` -- ``A = U diag(sigma) V^T``.  ``U`` is the orthonormal factor of a
  seeded m x n N(0,1) matrix with the signs fixed so that its triangular factor has a positive
  diagonal (Haar-distributed, the first n columns of the Haar matrix in Section 5.3, Eq. (5.2)),
  ``V`` the same for an n x n N(0,1) matrix, and ``sigma_i = kappa^{-(i-1)/(n-1)}`` (log-spaced
  from 1 to 1/kappa, the reading of ``gallery('randsvd', n, kappa)`` used throughout Section 5).
* ``usv_torch(m, n, kappa, seed, device)`` -- the same recipe drawn with torch's generator on the
  given device and orthonormalised with ``torch.linalg.qr`` (fast at m = 2^20 and above; its bits
  differ from ``usv``'s, so parity tests use ``usv`` and timing runs may use this one).
* ``coherent_diag(m, n, seed)`` -- the maximally coherent ``[D; 0]`` with D diagonal, the
  worst-coherence shape of Eq. (5.1) with a diagonal top block.  Without the smoothing transform
  an unsmoothed uniform sample misses some of the first n rows, so column j of the sample can be
  exactly zero.
* ``batch_manifest(count, seed)`` -- the heterogeneous batch: m log-uniform in [4096, 2^20],
  n uniform on {8,16,32,64,128}, s = 3n, kappa log-uniform in [1, 1e14].

Everything is drawn with numpy's PCG64 from the given seed.
"""
from __future__ import annotations

import numpy as np

__all__ = ["usv", "usv_factors", "usv_torch", "coherent_diag", "batch_manifest", "log_sigmas"]


def log_sigmas(n: int, kappa: float) -> np.ndarray:
    """sigma_i = kappa^{-(i-1)/(n-1)}, i = 1..n (sigma_1 = 1, sigma_n = 1/kappa)."""
    if n == 1:
        return np.ones(1)
    e = np.arange(n, dtype=np.float64) / (n - 1)
    return np.power(float(kappa), -e)


def _haar_columns(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def usv_factors(m: int, n: int, kappa: float, seed: int):
    """Return (U, sigma, V) for ``usv`` (U: m x n orthonormal, V: n x n orthogonal)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = _haar_columns(rng, m, n)
    v = _haar_columns(rng, n, n)
    return u, log_sigmas(n, kappa), v


def usv(m: int, n: int, kappa: float, seed: int, return_factors: bool = False):
    """A = U diag(sigma) V^T as a C-contiguous float64 array (see module docstring)."""
    u, s, v = usv_factors(m, n, kappa, seed)
    a = np.ascontiguousarray((u * s[None, :]) @ v.T)
    if return_factors:
        return a, (u, s, v)
    return a


def usv_torch(m: int, n: int, kappa: float, seed: int, device="cuda"):
    """A = U diag(sigma) V^T drawn with torch on `device` (float64, row-major)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def haar(rows, cols):
        x = torch.randn((rows, cols), generator=g, dtype=torch.float64, device=device)
        q, r = torch.linalg.qr(x, mode="reduced")
        del x
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        return q.mul_(d[None, :])

    u = haar(m, n)
    v = haar(n, n)
    s = torch.from_numpy(log_sigmas(n, kappa)).to(device)
    u.mul_(s[None, :])   # in place: at m = 2^23, n = 512 one copy is 34 GB
    return (u @ v.T).contiguous()


def coherent_diag(m: int, n: int, seed: int) -> np.ndarray:
    """[D; 0] with D = diag(d), d_i log-spaced in [1e-3, 1] in a seeded random order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.power(10.0, -3.0 * rng.random(n))
    a = np.zeros((m, n))
    a[np.arange(n), np.arange(n)] = d
    return a


def coherent_randsvd(m: int, n: int, kappa: float, seed: int) -> np.ndarray:
    """A = Q_A R_A with Q_A = [I_n; 0] and R_A an n x n matrix with singular values log-spaced from 1
    to 1/kappa and Haar singular vectors (the maximally coherent inputs of Section 5.1, Eq.
    e_ErrorRange; R_A plays the part of a randsvd matrix)."""
    a = np.zeros((m, n))
    a[:n] = usv(n, n, kappa, seed)
    return a


def batch_manifest(count: int = 512, seed: int = 20240617):
    """Seeded heterogeneous batch description: list of dicts (m, n, s, kappa, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        m = int(round(np.exp(rng.uniform(np.log(4096.0), np.log(1048576.0)))))
        n = int(rng.choice([8, 16, 32, 64, 128]))
        kappa = float(10.0 ** rng.uniform(0.0, 14.0))
        out.append({"m": m, "n": n, "s": 3 * n, "kappa": kappa, "seed": seed + 1 + i})
    return out
