"""GPU test of the autotuner: rpcholqr_autotune times the candidate launch parameters (the SPLIT64 first
pass's diagonal-block width and the Gram's split-K factor; the FP64 wide Gram's split-K factor) on
synthetic matrices, keeps the fastest per shape class, and writes the table that rpcholqr_plan_create
reads back.  Every candidate changes rounding only: a plan created from the table still matches the
oracle under the parity gates.
"""
import json

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("mode_name,shapes", [("SPLIT64", [(65536, 128, 384), (20000, 96, 288)]),
                                              ("FP64", [(30000, 256, 768)])])
def test_autotune_writes_a_table_the_plan_reads(lib, oracle_mod, tmp_path, mode_name, shapes):
    mode = getattr(lib, mode_name)
    max_m = max(x[0] for x in shapes)
    max_n = max(x[1] for x in shapes)
    max_s = max(x[2] for x in shapes)
    path = str(tmp_path / "tune.json")
    plan = lib.rpcholqr_plan_create(0, max_m, max_n, max_s, mode=mode)
    try:
        text = lib.rpcholqr_autotune(plan, shapes, reps=2, out_json=path)
    finally:
        plan.close()
    table = json.loads(open(path).read())
    assert json.loads(text) == table
    assert len(table["entries"]) == len(shapes)
    for e in table["entries"]:
        assert e["mode"] == {"SPLIT64": "split", "FP64": "fp64"}[mode_name] and e["ms"] > 0
        if mode_name == "SPLIT64":
            assert e["split_sub"] in (16, 32)
    assert lib.rpcholqr_autotune_parse(path) == len(shapes)
    # a plan created from the table: same results as the oracle under the usual gates
    tuned = lib.rpcholqr_plan_create(0, max_m, max_n, max_s, mode=mode, autotune_json=path)
    try:
        assert json.loads(lib.rpcholqr_autotune_table(tuned))["entries"] == table["entries"]
        m, n, s = shapes[0]
        A = inputs.usv(m, n, 1e8, 71)
        Q, R, info = lib.rpcholqr_factor(tuned, torch.from_numpy(A).to(DEV), s, 3)
        assert info.cpu().tolist() == [0, -1]
        o = oracle_mod.rpcholqr(A, s, 3)
        Rh = R.cpu().numpy()
        assert np.linalg.norm(Rh - o["R"], 2) <= 1e-12 * np.linalg.norm(o["R"], 2)
        orth = oracle_mod.orth_error_fast(Q.cpu().numpy())
        assert orth <= 10 * oracle_mod.orth_error_fast(o["Q"]) and orth <= 1e-13
    finally:
        tuned.close()
