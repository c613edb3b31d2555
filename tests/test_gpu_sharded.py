"""GPU tests of the row-sharded steps (one GPU: the blocks of two "processes" are emulated in one
process by calling the steps per block and doing the two exchanges by hand; the single-rank driver
runs over a one-process NCCL group).

Pins: the blocks' owned-row samples sum to exactly the sample rpcholqr_factor draws, so R_s is the
same bits as rpcholqr_sketch_r; the sharded factors match the oracle with the gates of the unsharded
tests; a one-rank run of the driver reproduces rpcholqr_factor bit for bit (same kernels, one Gram
part).
"""
import os
import socket

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def nrm2(x):
    return float(np.linalg.norm(x, 2))


@pytest.mark.parametrize("m,n,kappa,cuts", [(20011, 50, 1e8, (7000,)), (30000, 128, 1e12, (1, 15000, 29999)),
                                            (9000, 200, 1e6, (4500,))])
def test_sharded_steps_match_oracle(lib, oracle_mod, m, n, kappa, cuts):
    A = inputs.usv(m, n, kappa, 60 + n)
    s, seed = 3 * n, 13
    bounds = [0, *cuts, m]
    blocks = [(bounds[i], bounds[i + 1] - bounds[i]) for i in range(len(bounds) - 1)]
    plan = lib.rpcholqr_plan_create(0, m, n, s)
    try:
        Ad = cu(A)
        parts = [lib.rpcholqr_gather_owned_rows(Ad[o:o + ml], o, m, s, seed) for o, ml in blocks]
        # summing blocks that own disjoint rows is exact, in any order
        As = parts[0][0].clone()
        for p in parts[1:]:
            As += p[0]
        assert all(int(p[1][0]) == 0 for p in parts)
        Rs, info = lib.rpcholqr_sketch_r_from_sample(plan, As)
        assert int(info[0]) == 0
        Rs_ref, _ = lib.rpcholqr_sketch_r(plan, Ad, s, seed)
        assert torch.equal(Rs, Rs_ref)
        A1s, Gs = [], []
        for o, ml in blocks:
            A1, G, info = lib.rpcholqr_precondition_gram(plan, Ad[o:o + ml].contiguous(), Rs)
            assert int(info[0]) == 0
            A1s.append(A1)
            Gs.append(G)
        G = lib.rpcholqr_sum_partials(torch.stack(Gs).contiguous())
        R1, info = lib.rpcholqr_cholesky(plan, G)
        assert int(info[0]) == 0
        Q = torch.cat([lib.rpcholqr_solve_rows(plan, A1, R1, Y=A1)[0] for A1 in A1s])
        R = lib.rpcholqr_triu_mul(R1, Rs)
        o = oracle_mod.rpcholqr(A, s, seed)
        Qh, Rh = host(Q), host(R)
        assert nrm2(Rh - o["R"]) <= 1e-12 * nrm2(o["R"])
        if kappa <= 1e8:
            floor = nrm2(o["Q"] - oracle_mod.rpcholqr(A, s, seed, variant=1)["Q"])
            assert nrm2(Qh - o["Q"]) <= max(1e-10, 10 * floor)
        assert oracle_mod.orth_error(Qh) <= 10 * oracle_mod.orth_error(o["Q"])
    finally:
        plan.close()


def test_sum_partials_order_and_values(lib):
    rng = np.random.default_rng(1)
    P = rng.standard_normal((5, 33, 33))
    G = lib.rpcholqr_sum_partials(cu(P))
    ref = P[0].copy()
    for k in range(1, 5):
        ref += P[k]
    assert np.array_equal(host(G), ref)


def test_gather_owned_rows_rejects_bad_blocks(lib):
    A = torch.zeros((10, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_gather_owned_rows(A, 95, 100, 12, 1)     # block runs past m


def test_single_rank_driver_reproduces_factor(lib):
    import torch.distributed as dist
    from paper_2406_11751_gb300.sharded import CudaSteps, TorchDistComm, factor_row_sharded
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=DEV)
    try:
        m, n, s, seed = 50000, 96, 288, 3
        A = torch.from_numpy(inputs.usv(m, n, 1e10, 5)).to(DEV)
        plan = lib.rpcholqr_plan_create(0, m, n, s)
        try:
            Q, R, st = factor_row_sharded(CudaSteps(plan), TorchDistComm(), A, 0, m, s, seed)
            Q0, R0, info = lib.rpcholqr_factor(plan, A, s, seed)
            assert st == 0 and int(info[0]) == 0
            assert torch.equal(Q, Q0) and torch.equal(R, R0)
        finally:
            plan.close()
    finally:
        dist.destroy_process_group()
