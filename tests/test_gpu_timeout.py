"""Bounded device waits: a plan whose spin limit is one poll makes the tensor-core pipeline waits of the
SPLIT64 kernels give up, and the call reports RPCHOLQR_ERR_TIMEOUT in its device status word instead of
waiting.  Nothing is made to fault: the waits run out because their phase is not complete at the first
poll (the producers are still slicing).  Each kernel still waits for its own tensor-core work with the
default limit before it frees its tensor memory, so the same plan, back at the default limit, factors
the same matrix again and matches the oracle.
"""
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


def test_plan_options_roundtrip_and_reject_bad_values(lib):
    plan = lib.rpcholqr_plan_create(0, 4096, 16, 48)
    try:
        assert lib.rpcholqr_plan_get_option(plan, lib.OPT_SPIN_LIMIT) == 1 << 24
        assert lib.rpcholqr_plan_get_option(plan, lib.OPT_SCALE_SAMPLE) == 1
        assert lib.rpcholqr_plan_get_option(plan, lib.OPT_DETERMINISTIC) == 1
        lib.rpcholqr_plan_set_option(plan, lib.OPT_SPIN_LIMIT, 1000)
        assert lib.rpcholqr_plan_get_option(plan, lib.OPT_SPIN_LIMIT) == 1000
        for opt, val, code in ((lib.OPT_SPIN_LIMIT, 0, lib.ERR_ARG), (lib.OPT_SCALE_SAMPLE, 2, lib.ERR_ARG),
                               (lib.OPT_DETERMINISTIC, 0, lib.ERR_UNSUPPORTED), (99, 1, lib.ERR_ARG)):
            with pytest.raises(lib.RpcholqrError) as e:
                lib.rpcholqr_plan_set_option(plan, opt, val)
            assert e.value.code == code
    finally:
        plan.close()


def test_short_spin_limit_reports_timeout_then_recovers(lib, oracle_mod):
    m, n, s, seed = 65536, 128, 384, 3
    A = inputs.usv(m, n, 1e6, 77)
    Ad = cu(A)
    plan = lib.rpcholqr_plan_create(0, m, n, s, mode=lib.SPLIT64)
    try:
        lib.rpcholqr_plan_set_option(plan, lib.OPT_SPIN_LIMIT, 1)
        _, _, info = lib.rpcholqr_factor(plan, Ad, s, seed)
        assert info.cpu().tolist()[0] == lib.ERR_TIMEOUT
        # the split product alone, at the same limit
        X = cu(np.random.default_rng(1).standard_normal((20000, 64)))
        Y = cu(np.triu(np.random.default_rng(2).standard_normal((64, 64))))
        _, info = lib.rpcholqr_ozaki_gemm(plan, X, Y)
        assert info.cpu().tolist()[0] == lib.ERR_TIMEOUT
        # back to the default: the plan and the context are usable and the results match the oracle
        lib.rpcholqr_plan_set_option(plan, lib.OPT_SPIN_LIMIT, 1 << 24)
        Q, R, info = lib.rpcholqr_factor(plan, Ad, s, seed)
        assert info.cpu().tolist() == [0, -1]
        o = oracle_mod.rpcholqr(A, s, seed)
        Qh, Rh = host(Q), host(R)
        assert np.linalg.norm(Rh - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
        assert oracle_mod.orth_error(Qh) <= 10 * oracle_mod.orth_error(o["Q"])
    finally:
        plan.close()


def test_unscaled_sample_gives_the_same_factorisation(lib, oracle_mod):
    # R = R1 R_s does not depend on the sample's scale in exact arithmetic (Remark r_exp scales it only
    # to keep ||A1|| near 1): with the scale off, R and Q still match the oracle (which scales)
    m, n, s, seed = 20011, 50, 150, 4
    A = inputs.usv(m, n, 1e8, 78)
    for mode in (lib.FP64, lib.SPLIT64):
        plan = lib.rpcholqr_plan_create(0, m, n, s, mode=mode)
        try:
            lib.rpcholqr_plan_set_option(plan, lib.OPT_SCALE_SAMPLE, 0)
            Q, R, info = lib.rpcholqr_factor(plan, cu(A), s, seed)
            assert info.cpu().tolist() == [0, -1]
        finally:
            plan.close()
        o = oracle_mod.rpcholqr(A, s, seed)
        assert np.linalg.norm(host(R) - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
        assert oracle_mod.orth_error(host(Q)) <= 10 * oracle_mod.orth_error(o["Q"])
