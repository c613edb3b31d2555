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
        # second call: other shape, same scratch; third: fewer rows than one 256-row panel
        cases = [(30011, 64, 1e8, 1), (4099, 37, 1e3, 2), (200, 40, 1e4, 3)]
        for k, (m, n, kappa, seed) in enumerate(cases):
            A = inputs.usv(m, n, kappa, 500 + seed)
            Rs = oracle_mod.rpcholqr(A, 3 * n, seed)["Rs"]
            Ad, Rsd = _cu(A), _cu(Rs)
            A1_ref, G_ref, info_ref = lib.rpcholqr_precondition_gram(plan, Ad, Rsd)
            A1 = torch.full((m, n), np.nan, dtype=torch.float64, device=DEV)
            G = torch.full((n, n), np.nan, dtype=torch.float64, device=DEV)
            info = torch.empty(2, dtype=torch.int32, device=DEV)
            torch.cuda.synchronize()
            free0, torch0 = torch.cuda.mem_get_info(DEV)[0], torch.cuda.memory_allocated(DEV)
            lib.rpcholqr_precondition_gram_noalloc(Ad, Rsd, A1, G, info)
            torch.cuda.synchronize()
            if k > 0:
                # after the first call (which looks up the scratch address) a call allocates nothing:
                # neither through torch's allocator nor from the device's free memory
                assert torch.cuda.memory_allocated(DEV) == torch0
                assert torch.cuda.mem_get_info(DEV)[0] == free0
            assert info.cpu().tolist() == info_ref.cpu().tolist() == [0, -1]
            assert _rel(A1, A1_ref) <= 1e-13
            assert _rel(G, G_ref) <= 1e-13
    finally:
        plan.close()


def test_noalloc_rejects_mismatched_buffers(lib):
    # the wrapper checks every caller buffer before the call: a short A1, a G with the wrong leading
    # dimension, a non-contiguous Rs or a missing info would otherwise be written past their ends
    m, n = 1000, 16
    A = torch.zeros((m, n), dtype=torch.float64, device=DEV)
    Rs = torch.eye(n, dtype=torch.float64, device=DEV)
    A1 = torch.empty_like(A)
    G = torch.empty((n, n), dtype=torch.float64, device=DEV)
    info = torch.empty(2, dtype=torch.int32, device=DEV)
    bad = [
        dict(A1=A1[: m - 1]),
        dict(G=torch.empty((n, n + 3), dtype=torch.float64, device=DEV)[:, :n]),
        dict(Rs=torch.eye(2 * n, dtype=torch.float64, device=DEV)[:n, :n]),
        dict(info=None),
        dict(info=torch.empty(1, dtype=torch.int32, device=DEV)),
        dict(info=torch.empty(2, dtype=torch.int64, device=DEV)),
    ]
    for override in bad:
        args = dict(A1=A1, G=G, Rs=Rs, info=info)
        args.update(override)
        with pytest.raises((ValueError, TypeError)):
            lib.rpcholqr_precondition_gram_noalloc(A, args["Rs"], args["A1"], args["G"], args["info"])


def test_noalloc_rejects_n_beyond_scratch(lib):
    A = torch.zeros((1000, 65), dtype=torch.float64, device=DEV)
    Rs = torch.eye(65, dtype=torch.float64, device=DEV)
    A1 = torch.empty_like(A)
    G = torch.empty((65, 65), dtype=torch.float64, device=DEV)
    info = torch.empty(2, dtype=torch.int32, device=DEV)
    with pytest.raises(lib.RpcholqrError) as e:
        lib.rpcholqr_precondition_gram_noalloc(A, Rs, A1, G, info)
    assert e.value.code == 8   # RPCHOLQR_ERR_UNSUPPORTED
