"""The allocation-free entry point (rpcholqr_precondition_gram_noalloc) against the plan-based one.

Callers that may not allocate device memory while running (framework-owned allocators, services
that reserve memory up front) use the no-alloc variant, whose scratch is a fixed device array in
the library.  Its results must equal the plan-based rpcholqr_precondition_gram within the tolerance
the parity tests use, on two calls in a row (the second call reuses the scratch the first left).
This file is named to run last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(torch.linalg.matrix_norm(a - b, 2) / torch.linalg.matrix_norm(b, 2))


def test_noalloc_matches_plan_entry_point_twice(lib, oracle_mod):
    plan = lib.rpcholqr_plan_create(0, 40000, 64, 192)
    try:
        cases = [(30011, 64, 1e8, 1), (4099, 37, 1e3, 2)]   # second call: other shape, same scratch
        for m, n, kappa, seed in cases:
            A = inputs.usv(m, n, kappa, 500 + seed)
            Rs = oracle_mod.rpcholqr(A, 3 * n, seed)["Rs"]
            Ad, Rsd = _cu(A), _cu(Rs)
            A1_ref, G_ref, info_ref = lib.rpcholqr_precondition_gram(plan, Ad, Rsd)
            A1 = torch.full((m, n), np.nan, dtype=torch.float64, device=DEV)
            G = torch.full((n, n), np.nan, dtype=torch.float64, device=DEV)
            info = torch.empty(2, dtype=torch.int32, device=DEV)
            lib.rpcholqr_precondition_gram_noalloc(Ad, Rsd, A1, G, info)
            torch.cuda.synchronize()
            assert info.cpu().tolist() == info_ref.cpu().tolist() == [0, -1]
            assert _rel(A1, A1_ref) <= 1e-13
            assert _rel(G, G_ref) <= 1e-13
    finally:
        plan.close()


def test_noalloc_rejects_n_beyond_scratch(lib):
    A = torch.zeros((1000, 65), dtype=torch.float64, device=DEV)
    Rs = torch.eye(65, dtype=torch.float64, device=DEV)
    A1 = torch.empty_like(A)
    G = torch.empty((65, 65), dtype=torch.float64, device=DEV)
    info = torch.empty(2, dtype=torch.int32, device=DEV)
    with pytest.raises(lib.RpcholqrError) as e:
        lib.rpcholqr_precondition_gram_noalloc(A, Rs, A1, G, info)
    assert e.value.code == 8   # RPCHOLQR_ERR_UNSUPPORTED
