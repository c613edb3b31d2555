"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/rpcholqr.h
declares (no GPU needed: only host-only entry points are called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rpcholqr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rpcholqr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rpcholqr_plan_create", "rpcholqr_plan_destroy", "rpcholqr_factor",
                 "rpcholqr_factor_host", "rpcholqr_workspace_size"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = lib.load_library()
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib.EXPORTED_SYMBOLS) <= set(declared_functions())


def test_host_only_entry_points(lib):
    assert lib.rpcholqr_status_string(4) == "RPCHOLQR_ERR_NOT_SPD"
    assert lib.rpcholqr_status_string(99) == "RPCHOLQR_UNKNOWN_STATUS"
    b = lib.rpcholqr_workspace_size(1 << 20, 128, 384)
    assert b >= 8 * (384 * 128 + 4 * 128 * 128 + 152 * 128 * 128)
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_workspace_size(100, 0, 10)         # n < 1
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_workspace_size(10000, 2049, 6200)   # n above the built maximum
    # wide panels keep at most one Gram partial per 1024 rows and at most 1 GiB of them
    wide = lib.rpcholqr_workspace_size(6000, 2048, 6000)
    assert 8 * 6 * 2048 * 2048 <= wide <= 8 * (6000 * 2048 + 13 * 2048 * 2048)
    with pytest.raises(lib.RpcholqrError):
        lib.rpcholqr_workspace_size(100, 10, 5)         # s < n
    h = ctypes.c_void_p()
    assert lib.load_library().rpcholqr_plan_create(ctypes.byref(h), 0, 0, 100, 0, 10, None) == 1
    assert lib.load_library().rpcholqr_plan_create(ctypes.byref(h), 0, 7, 100, 10, 30, None) in (1, 8)
    # an unreadable tuning table is refused before any device work
    assert lib.load_library().rpcholqr_plan_create(ctypes.byref(h), 0, 0, 1000, 10, 30, b"{nope") == 1
    assert lib.load_library().rpcholqr_plan_destroy(None) == 0


def test_kernels_are_built_for_sm103a(lib):
    # the fatbin must carry sm_103a code; checked from the build flags, not by disassembly
    import importlib
    b = importlib.import_module("paper_2406_11751_gb300.build")
    assert b.ARCH_FLAGS == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(b.LIB_PATH)


def test_autotune_table_parser(lib, tmp_path):
    table = """{"gpu": "x", "sms": 152, "entries": [
        {"mode": "split", "np": 128, "m_log2": 20, "split_sub": 16, "gram_ranges": 38, "syrk_ranges": 0,
         "ms": 12.5},
        {"m_log2": 23, "np": 512, "mode": "fp64", "syrk_ranges": 8}]}"""
    assert lib.rpcholqr_autotune_parse(table) == 2
    path = tmp_path / "tune.json"
    path.write_text(table)
    assert lib.rpcholqr_autotune_parse(str(path)) == 2
    assert lib.rpcholqr_autotune_parse('{"entries": []}') == 0
    for bad in ('{"entries": [{"np": 128, "m_log2": 20}]}',              # no mode
                '{"entries": [{"mode": "fp16", "np": 128, "m_log2": 20}]}',
                '{"entries": [{"mode": "split", "np": 128, "m_log2": 20, "split_sub": -1}]}',
                '{"no_entries": 1}', str(tmp_path / "missing.json")):
        with pytest.raises(lib.RpcholqrError):
            lib.rpcholqr_autotune_parse(bad)
