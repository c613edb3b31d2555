"""rpCholesky-QR on GB300 (sm_103a): thin Python binding over ``librpcholqr.so``.

Garrison & Ipsen, "A randomized preconditioned Cholesky-QR algorithm" (arXiv 2406.11751),
Algorithm alg_2 (Section 4).  Every arithmetic step runs in the library's CUDA kernels; this module
only marshals torch tensors (device memory, streams) into the C ABI of ``include/rpcholqr.h`` and
keeps the same function names.  There is no CPU fallback: if the library is missing or a tensor is
not on a CUDA device the call raises.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH, build  # noqa: F401  (re-exported for __graft_entry__)

__all__ = [
    "RpcholqrError", "Plan", "STATUS", "load_library", "rpcholqr_plan_create", "rpcholqr_plan_destroy",
    "rpcholqr_workspace_size", "rpcholqr_factor", "rpcholqr_factor_host", "rpcholqr_sample_indices",
    "rpcholqr_sketch_r", "rpcholqr_precondition_gram", "rpcholqr_cholesky", "rpcholqr_solve_rows",
    "rpcholqr_triu_mul", "rpcholqr_probe_fp64_mma", "rpcholqr_status_string", "EXPORTED_SYMBOLS",
    "rpcholqr_plan_enable_timing", "rpcholqr_plan_collect_timing", "PHASES", "rpcholqr_ozaki_gemm",
    "rpcholqr_ozaki_gram", "SPLIT64", "rpcholqr_cholqr", "rpcholqr_cholqr2", "Batch",
    "rpcholqr_batch_create", "rpcholqr_batch_destroy", "rpcholqr_batch_factor", "rpcholqr_factor_batched",
    "rpcholqr_batch_capture",
    "rpcholqr_batch_replay", "rpcholqr_batch_autotune", "FP32", "rpcholqr_factor_f32",
    "rpcholqr_gather_owned_rows", "rpcholqr_sketch_r_from_sample", "rpcholqr_sum_partials",
    "rpcholqr_plan_set_smoothing", "rpcholqr_smoothed_sample", "SMOOTH_NONE", "SMOOTH_WHT", "SMOOTH_DCT",
    "rpcholqr_plan_split_pass2_fp64", "rpcholqr_scholqr3", "rpcholqr_ozaki_update",
]

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NONFINITE", 3: "ERR_SINGULAR_SKETCH", 4: "ERR_NOT_SPD",
          5: "ERR_TIMEOUT", 6: "ERR_CUDA", 7: "ERR_NOMEM", 8: "ERR_UNSUPPORTED"}
OK, ERR_ARG, ERR_NONFINITE, ERR_SINGULAR_SKETCH, ERR_NOT_SPD = 0, 1, 2, 3, 4
FP64 = 0
SPLIT64 = 1
FP32 = 2
SMOOTH_NONE, SMOOTH_WHT, SMOOTH_DCT = 0, 1, 2
OPT_SPIN_LIMIT, OPT_SCALE_SAMPLE, OPT_DETERMINISTIC, OPT_BATCH_CAPACITY, OPT_IMAGE_ROWS = 0, 1, 2, 3, 4
ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM, ERR_UNSUPPORTED = 5, 6, 7, 8
MAX_N = 2048

EXPORTED_SYMBOLS = (
    "rpcholqr_plan_create", "rpcholqr_plan_destroy", "rpcholqr_workspace_size", "rpcholqr_factor",
    "rpcholqr_factor_host", "rpcholqr_sample_indices", "rpcholqr_sketch_r",
    "rpcholqr_precondition_gram", "rpcholqr_cholesky", "rpcholqr_solve_rows", "rpcholqr_triu_mul",
    "rpcholqr_probe_fp64_mma", "rpcholqr_status_string", "rpcholqr_plan_enable_timing",
    "rpcholqr_plan_collect_timing", "rpcholqr_ozaki_gemm", "rpcholqr_ozaki_gram", "rpcholqr_cholqr",
    "rpcholqr_cholqr2", "rpcholqr_batch_create", "rpcholqr_batch_destroy", "rpcholqr_batch_factor",
    "rpcholqr_factor_batched",
    "rpcholqr_batch_capture", "rpcholqr_batch_replay", "rpcholqr_batch_autotune", "rpcholqr_factor_f32",
    "rpcholqr_gather_owned_rows", "rpcholqr_sketch_r_from_sample", "rpcholqr_sum_partials",
    "rpcholqr_plan_set_smoothing", "rpcholqr_smoothed_sample", "rpcholqr_plan_split_pass2_fp64",
    "rpcholqr_scholqr3", "rpcholqr_plan_set_option", "rpcholqr_plan_get_option",
    "rpcholqr_factor_batched", "rpcholqr_batch_factor", "rpcholqr_plan_collect_kernel_timing",
    "rpcholqr_autotune", "rpcholqr_autotune_table", "rpcholqr_autotune_parse", "rpcholqr_ozaki_update",
)
PHASES = ("sample", "sketch_qr", "prep_rs", "pass1", "pass1_update", "pass1_solve2", "gram_reduce",
          "cholesky", "prep_r1", "pass2", "recover_r")
KERNEL_CLASSES = ("rowpass", "split_update", "split_gemm_sub", "split_gemm", "split_gram", "fp64_gemm",
                  "fp64_syrk", "sketch_qr", "cholesky")


class RpcholqrError(RuntimeError):
    """A host-side (argument / launch / allocation) error returned by the C ABI."""

    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)}")
        self.code = code


_lib = None


def load_library():
    """Load librpcholqr.so (no automatic build: a missing library is an error)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           f"`python -m paper_2406_11751_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                           ctypes.c_double)
    st = ctypes.c_int
    sig = {
        "rpcholqr_plan_create": [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, I64, I32, I32, ctypes.c_char_p],
        "rpcholqr_autotune": [P, I32, P, P, P, I32, ctypes.c_char_p],
        "rpcholqr_autotune_table": [P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
        "rpcholqr_autotune_parse": [ctypes.c_char_p, ctypes.POINTER(I32)],
        "rpcholqr_plan_destroy": [P],
        "rpcholqr_plan_set_option": [P, I32, I64],
        "rpcholqr_plan_get_option": [P, I32, ctypes.POINTER(I64)],
        "rpcholqr_workspace_size": [P, I64, I32, I32, ctypes.POINTER(ctypes.c_size_t)],
        "rpcholqr_factor": [P, P, I64, I32, I64, I32, U64, P, I64, P, P, P],
        "rpcholqr_factor_host": [P, P, I64, I32, I64, I32, U64, P, I64, P, P, P],
        "rpcholqr_factor_f32": [P, P, I64, I32, I64, I32, U64, P, I64, P, P, P],
        "rpcholqr_gather_owned_rows": [P, I64, I32, I64, I64, I64, I32, U64, P, I64, P, P],
        "rpcholqr_sketch_r_from_sample": [P, P, I32, I32, I64, P, P, P],
        "rpcholqr_sum_partials": [P, I32, I32, P, P],
        "rpcholqr_plan_set_smoothing": [P, I32],
        "rpcholqr_plan_split_pass2_fp64": [P, ctypes.POINTER(I32)],
        "rpcholqr_smoothed_sample": [P, P, I64, I32, I64, I32, U64, P, I64, P, P],
        "rpcholqr_sample_indices": [U64, U64, I64, I32, P, P],
        "rpcholqr_sketch_r": [P, P, I64, I32, I64, I32, U64, P, P, P],
        "rpcholqr_precondition_gram": [P, P, I64, I32, I64, P, P, I64, P, P, P],
        "rpcholqr_cholesky": [P, P, I32, P, P, P],
        "rpcholqr_solve_rows": [P, P, I64, I32, I64, P, P, I64, P, P],
        "rpcholqr_triu_mul": [P, P, I32, P, P],
        "rpcholqr_probe_fp64_mma": [ctypes.c_int, I32, ctypes.POINTER(D)],
        "rpcholqr_plan_enable_timing": [P, I32],
        "rpcholqr_plan_collect_timing": [P, P, ctypes.POINTER(I32), ctypes.POINTER(I64)],
        "rpcholqr_plan_collect_kernel_timing": [P, P, P, P],
        "rpcholqr_ozaki_gemm": [P, P, I64, I32, I64, P, I32, I64, P, I64, P, P],
        "rpcholqr_ozaki_update": [P, P, I64, I32, I64, P, I32, I64, P, I64, P, I64, P, P],
        "rpcholqr_ozaki_gram": [P, P, I64, I32, I64, P, P, P],
        "rpcholqr_cholqr": [P, P, I64, I32, I64, P, I64, P, P, P],
        "rpcholqr_cholqr2": [P, P, I64, I32, I64, P, I64, P, P, P],
        "rpcholqr_scholqr3": [P, P, I64, I32, I64, P, I64, P, P, P],
        "rpcholqr_batch_create": [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, I64, I32, I32, I32],
        "rpcholqr_batch_destroy": [P],
        "rpcholqr_batch_factor": [P, I32, P, P, P, P, P, P, P, P, P, P, P],
        "rpcholqr_factor_batched": [P, I32, P, P, P, P, P, P, P, P, P, P, P],
        "rpcholqr_batch_capture": [P, I32, P, P, P, P, P, P, P, P, P, P, P],
        "rpcholqr_batch_replay": [P, P],
        "rpcholqr_batch_autotune": [P, I32, P, P, P, P, P, P, P, P, P, P, I32, ctypes.POINTER(I32),
                                    ctypes.POINTER(ctypes.c_float), P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = st
    lib.rpcholqr_status_string.argtypes = [ctypes.c_int]
    lib.rpcholqr_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(fn: str, code: int):
    if code != 0:
        raise RpcholqrError(fn, code)


def rpcholqr_status_string(code: int) -> str:
    return load_library().rpcholqr_status_string(int(code)).decode()


# ---- tensor helpers -----------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _mat(x, name, dtype=None):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D row-major tensor with unit column stride")
    if x.dtype != (dtype or torch.float64):
        raise TypeError(f"{name} must be {dtype or torch.float64}")
    return x


def _stream(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owner of a C plan handle (device workspace for matrices up to max_m x max_n, max_s samples)."""

    def __init__(self, handle, device, max_m, max_n, max_s):
        self.handle = handle
        self.device = device
        self.max_m, self.max_n, self.max_s = max_m, max_n, max_s

    def close(self):
        if self.handle:
            load_library().rpcholqr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rpcholqr_plan_create(device: int, max_m: int, max_n: int, max_s: int, mode: int = FP64,
                         autotune_json: str = None) -> Plan:
    """A plan; autotune_json (optional): a tuning table from rpcholqr_autotune, as JSON text or a path."""
    h = ctypes.c_void_p()
    tj = autotune_json.encode() if autotune_json is not None else None
    _check("rpcholqr_plan_create",
           load_library().rpcholqr_plan_create(ctypes.byref(h), device, mode, max_m, max_n, max_s, tj))
    return Plan(h, device, max_m, max_n, max_s)


def rpcholqr_autotune(plan: Plan, shapes, reps: int = 2, out_json: str = None) -> str:
    """Time the candidate launch parameters for each (m, n, s) of `shapes` (synthetic matrices), keep the
    fastest in the plan's table, write it to out_json if given; returns the table as JSON text."""
    k = len(shapes)
    ms = (ctypes.c_int64 * k)(*[int(x[0]) for x in shapes])
    ns = (ctypes.c_int32 * k)(*[int(x[1]) for x in shapes])
    ss = (ctypes.c_int32 * k)(*[int(x[2]) for x in shapes])
    lib = load_library()
    _check("rpcholqr_autotune", lib.rpcholqr_autotune(
        plan.handle, k, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(ns, ctypes.c_void_p),
        ctypes.cast(ss, ctypes.c_void_p), reps, out_json.encode() if out_json else None))
    return rpcholqr_autotune_table(plan)


def rpcholqr_autotune_table(plan: Plan) -> str:
    n = ctypes.c_size_t()
    lib = load_library()
    _check("rpcholqr_autotune_table", lib.rpcholqr_autotune_table(plan.handle, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check("rpcholqr_autotune_table", lib.rpcholqr_autotune_table(plan.handle, buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def rpcholqr_autotune_parse(json_or_path: str) -> int:
    """Number of entries of a tuning table (host-only check; raises on an unreadable table)."""
    k = ctypes.c_int32()
    _check("rpcholqr_autotune_parse", load_library().rpcholqr_autotune_parse(json_or_path.encode(), ctypes.byref(k)))
    return int(k.value)


def rpcholqr_plan_destroy(plan: Plan):
    plan.close()


def rpcholqr_plan_set_option(plan: Plan, option: int, value: int):
    """Set a plan option (OPT_SPIN_LIMIT, OPT_SCALE_SAMPLE, OPT_DETERMINISTIC, OPT_BATCH_CAPACITY, OPT_IMAGE_ROWS)."""
    _check("rpcholqr_plan_set_option", load_library().rpcholqr_plan_set_option(plan.handle, option, int(value)))


def rpcholqr_plan_get_option(plan: Plan, option: int) -> int:
    v = ctypes.c_int64()
    _check("rpcholqr_plan_get_option", load_library().rpcholqr_plan_get_option(plan.handle, option, ctypes.byref(v)))
    return int(v.value)


def rpcholqr_workspace_size(max_m: int, max_n: int, max_s: int, plan: Plan = None) -> int:
    """Bytes of device workspace a plan with these limits allocates (plan: its mode and device; None: an
    FP64 plan on a 152-SM GPU)."""
    b = ctypes.c_size_t()
    _check("rpcholqr_workspace_size", load_library().rpcholqr_workspace_size(
        plan.handle if plan is not None else None, max_m, max_n, max_s, ctypes.byref(b)))
    return int(b.value)


def _info(info, device):
    torch = _torch()
    if info is None:
        info = torch.empty(2, dtype=torch.int32, device=device)
    return info


def rpcholqr_factor(plan: Plan, A, s: int, seed: int, Q=None, R=None, info=None, stream=None):
    """(Q, R, info) of rpCholesky-QR; info is a device int32[2] {status, pivot} (not synchronised)."""
    torch = _torch()
    _mat(A, "A")
    m, n = A.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, device=A.device)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=A.device)
    _mat(Q, "Q")
    _mat(R, "R")
    info = _info(info, A.device)
    _check("rpcholqr_factor", load_library().rpcholqr_factor(
        plan.handle, _ptr(A), m, n, A.stride(0), s, seed, _ptr(Q), Q.stride(0), _ptr(R), _ptr(info),
        _stream(stream, A.device)))
    return Q, R, info


def rpcholqr_factor_f32(plan: Plan, A, s: int, seed: int, Q=None, R=None, info=None, stream=None):
    """(Q, R, info) of the FP32 mode (float32 A, Q, R; an FP32 plan); info as in rpcholqr_factor."""
    torch = _torch()
    _mat(A, "A", torch.float32)
    m, n = A.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float32, device=A.device)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float32, device=A.device)
    _mat(Q, "Q", torch.float32)
    _mat(R, "R", torch.float32)
    info = _info(info, A.device)
    _check("rpcholqr_factor_f32", load_library().rpcholqr_factor_f32(
        plan.handle, _ptr(A), m, n, A.stride(0), s, seed, _ptr(Q), Q.stride(0), _ptr(R), _ptr(info),
        _stream(stream, A.device)))
    return Q, R, info


def rpcholqr_gather_owned_rows(A_local, row_offset: int, m: int, s: int, seed: int, As=None, info=None,
                               stream=None, device=None):
    """The rows of the global s-row sample owned by the row block A_local (m_local x n, global rows
    row_offset ..), zeros elsewhere: (As (s x n), info)."""
    torch = _torch()
    _mat(A_local, "A_local")
    m_local, n = A_local.shape
    dev = A_local.device
    if As is None:
        As = torch.empty((s, n), dtype=torch.float64, device=dev)
    _mat(As, "As")
    info = _info(info, dev)
    _check("rpcholqr_gather_owned_rows", load_library().rpcholqr_gather_owned_rows(
        _ptr(A_local) if m_local else None, m_local, n, A_local.stride(0) if m_local else n, row_offset, m, s,
        seed, _ptr(As), As.stride(0), _ptr(info), _stream(stream, dev)))
    return As, info


def rpcholqr_sketch_r_from_sample(plan: Plan, As, Rs=None, info=None, stream=None):
    """R_s (n x n) of a gathered s x n sample: (Rs, info)."""
    torch = _torch()
    _mat(As, "As")
    s, n = As.shape
    if Rs is None:
        Rs = torch.empty((n, n), dtype=torch.float64, device=As.device)
    _mat(Rs, "Rs")
    info = _info(info, As.device)
    _check("rpcholqr_sketch_r_from_sample", load_library().rpcholqr_sketch_r_from_sample(
        plan.handle, _ptr(As), s, n, As.stride(0), _ptr(Rs), _ptr(info), _stream(stream, As.device)))
    return Rs, info


def rpcholqr_sum_partials(parts, G=None, stream=None):
    """G = parts[0] + parts[1] + ... (in that order) for a contiguous (k, n, n) tensor."""
    torch = _torch()
    if not isinstance(parts, torch.Tensor) or not parts.is_cuda or parts.dim() != 3 or not parts.is_contiguous() \
            or parts.dtype != torch.float64:
        raise TypeError("parts must be a contiguous float64 CUDA tensor of shape (k, n, n)")
    k, n, _ = parts.shape
    if G is None:
        G = torch.empty((n, n), dtype=torch.float64, device=parts.device)
    _mat(G, "G")
    _check("rpcholqr_sum_partials", load_library().rpcholqr_sum_partials(
        _ptr(parts), k, n, _ptr(G), _stream(stream, parts.device)))
    return G


def rpcholqr_plan_set_smoothing(plan: Plan, kind: int = SMOOTH_WHT):
    """Sample the smoothed F A (kind 1 Walsh-Hadamard, 2 cosine) or A itself (kind 0) on this plan."""
    _check("rpcholqr_plan_set_smoothing", load_library().rpcholqr_plan_set_smoothing(plan.handle, kind))


def rpcholqr_plan_split_pass2_fp64(plan: Plan) -> bool:
    """Whether the last split factorisation on plan took the FP64 second pass (synchronises)."""
    v = ctypes.c_int32()
    _check("rpcholqr_plan_split_pass2_fp64",
           load_library().rpcholqr_plan_split_pass2_fp64(plan.handle, ctypes.byref(v)))
    return bool(v.value)


def rpcholqr_smoothed_sample(plan: Plan, A, s: int, seed: int, As=None, info=None, stream=None):
    """(A_s, info): the s x n smoothed sample sqrt(m'/s) (F A)(idx, :) (smoothing enabled on plan)."""
    torch = _torch()
    _mat(A, "A")
    m, n = A.shape
    if As is None:
        As = torch.empty((s, n), dtype=torch.float64, device=A.device)
    _mat(As, "As")
    info = _info(info, A.device)
    _check("rpcholqr_smoothed_sample", load_library().rpcholqr_smoothed_sample(
        plan.handle, _ptr(A), m, n, A.stride(0), s, seed, _ptr(As), As.stride(0), _ptr(info),
        _stream(stream, A.device)))
    return As, info


def rpcholqr_factor_host(plan: Plan, A, s: int, seed: int, Q=None, R=None, stream=None):
    """Host-buffer variant: A, Q, R are CPU float64 tensors (pinned for full copy speed).
    Returns (Q, R, status, pivot) after the device work and the copies finished."""
    torch = _torch()
    if A.is_cuda or A.dtype != torch.float64 or A.dim() != 2 or A.stride(1) != 1:
        raise TypeError("A must be a row-major float64 CPU tensor")
    m, n = A.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    info = (ctypes.c_int32 * 2)()
    dev = torch.device("cuda", plan.device)
    _check("rpcholqr_factor_host", load_library().rpcholqr_factor_host(
        plan.handle, _ptr(A), m, n, A.stride(0), s, seed, _ptr(Q), Q.stride(0), _ptr(R),
        ctypes.cast(info, ctypes.c_void_p), _stream(stream, dev)))
    return Q, R, int(info[0]), int(info[1])


def rpcholqr_sample_indices(seed: int, m: int, s: int, stream_id: int = 0, idx=None, device=None,
                            stream=None):
    torch = _torch()
    if idx is None:
        idx = torch.empty(s, dtype=torch.int64, device=device if device is not None else "cuda")
    _check("rpcholqr_sample_indices", load_library().rpcholqr_sample_indices(
        seed, stream_id, m, s, _ptr(idx), _stream(stream, idx.device)))
    return idx


def rpcholqr_sketch_r(plan: Plan, A, s: int, seed: int, Rs=None, info=None, stream=None):
    torch = _torch()
    _mat(A, "A")
    m, n = A.shape
    if Rs is None:
        Rs = torch.empty((n, n), dtype=torch.float64, device=A.device)
    info = _info(info, A.device)
    _check("rpcholqr_sketch_r", load_library().rpcholqr_sketch_r(
        plan.handle, _ptr(A), m, n, A.stride(0), s, seed, _ptr(Rs), _ptr(info),
        _stream(stream, A.device)))
    return Rs, info


def rpcholqr_precondition_gram(plan: Plan, A, Rs, A1=None, G=None, info=None, stream=None):
    torch = _torch()
    _mat(A, "A")
    m, n = A.shape
    Rs = _mat(Rs.contiguous(), "Rs")
    if A1 is None:
        A1 = torch.empty((m, n), dtype=torch.float64, device=A.device)
    if G is None:
        G = torch.empty((n, n), dtype=torch.float64, device=A.device)
    info = _info(info, A.device)
    _check("rpcholqr_precondition_gram", load_library().rpcholqr_precondition_gram(
        plan.handle, _ptr(A), m, n, A.stride(0), _ptr(Rs), _ptr(A1), A1.stride(0), _ptr(G),
        _ptr(info), _stream(stream, A.device)))
    return A1, G, info


def rpcholqr_cholesky(plan: Plan, G, R1=None, info=None, stream=None):
    torch = _torch()
    G = _mat(G.contiguous(), "G")
    n = G.shape[0]
    if R1 is None:
        R1 = torch.empty((n, n), dtype=torch.float64, device=G.device)
    info = _info(info, G.device)
    _check("rpcholqr_cholesky", load_library().rpcholqr_cholesky(
        plan.handle, _ptr(G), n, _ptr(R1), _ptr(info), _stream(stream, G.device)))
    return R1, info


def rpcholqr_solve_rows(plan: Plan, X, T, Y=None, info=None, stream=None):
    torch = _torch()
    _mat(X, "X")
    m, n = X.shape
    T = _mat(T.contiguous(), "T")
    if Y is None:
        Y = torch.empty((m, n), dtype=torch.float64, device=X.device)
    info = _info(info, X.device)
    _check("rpcholqr_solve_rows", load_library().rpcholqr_solve_rows(
        plan.handle, _ptr(X), m, n, X.stride(0), _ptr(T), _ptr(Y), Y.stride(0), _ptr(info),
        _stream(stream, X.device)))
    return Y, info


def rpcholqr_triu_mul(R1, Rs, R=None, stream=None):
    torch = _torch()
    R1 = _mat(R1.contiguous(), "R1")
    Rs = _mat(Rs.contiguous(), "Rs")
    n = R1.shape[0]
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=R1.device)
    _check("rpcholqr_triu_mul", load_library().rpcholqr_triu_mul(
        _ptr(R1), _ptr(Rs), n, _ptr(R), _stream(stream, R1.device)))
    return R


def _cholqr_call(name, plan, A, Q, R, info, stream):
    torch = _torch()
    _mat(A, "A")
    m, n = A.shape
    if Q is None:
        Q = torch.empty((m, n), dtype=torch.float64, device=A.device)
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, device=A.device)
    info = _info(info, A.device)
    _check(name, getattr(load_library(), name)(
        plan.handle, _ptr(A), m, n, A.stride(0), _ptr(Q), Q.stride(0), _ptr(R), _ptr(info),
        _stream(stream, A.device)))
    return Q, R, info


def rpcholqr_cholqr(plan: Plan, A, Q=None, R=None, info=None, stream=None):
    """Basic Cholesky-QR (Algorithm alg_0) on the GPU; (Q, R, info)."""
    return _cholqr_call("rpcholqr_cholqr", plan, A, Q, R, info, stream)


def rpcholqr_cholqr2(plan: Plan, A, Q=None, R=None, info=None, stream=None):
    """Cholesky-QR2 on the GPU (the paper's comparison method); (Q, R, info)."""
    return _cholqr_call("rpcholqr_cholqr2", plan, A, Q, R, info, stream)


def rpcholqr_scholqr3(plan: Plan, A, Q=None, R=None, info=None, stream=None):
    """Shifted Cholesky-QR3 on the GPU (cited in Section 1 as the remedy for Cholesky-QR2's breakdown)."""
    return _cholqr_call("rpcholqr_scholqr3", plan, A, Q, R, info, stream)


def rpcholqr_ozaki_gemm(plan: Plan, X, Y, C=None, info=None, stream=None):
    """C = X Y as a split-precision (FP64-accurate) BF16 tensor-core product (SPLIT64 plan)."""
    torch = _torch()
    _mat(X, "X")
    _mat(Y, "Y")
    m, K = X.shape
    N = Y.shape[1]
    if C is None:
        C = torch.empty((m, N), dtype=torch.float64, device=X.device)
    info = _info(info, X.device)
    _check("rpcholqr_ozaki_gemm", load_library().rpcholqr_ozaki_gemm(
        plan.handle, _ptr(X), m, K, X.stride(0), _ptr(Y), N, Y.stride(0), _ptr(C), C.stride(0),
        _ptr(info), _stream(stream, X.device)))
    return C, info


def rpcholqr_ozaki_update(plan: Plan, X, Y, B, C=None, info=None, stream=None):
    """C = B - X Y with the split-precision (FP64-accurate) product (SPLIT64 plan); C may be B."""
    torch = _torch()
    _mat(X, "X")
    _mat(Y, "Y")
    _mat(B, "B")
    m, K = X.shape
    N = Y.shape[1]
    if tuple(B.shape) != (m, N):
        raise ValueError(f"B must be {m} x {N}, got {tuple(B.shape)}")
    if C is None:
        C = torch.empty((m, N), dtype=torch.float64, device=X.device)
    _mat(C, "C")
    if tuple(C.shape) != (m, N):
        raise ValueError(f"C must be {m} x {N}, got {tuple(C.shape)}")
    info = _info(info, X.device)
    _check("rpcholqr_ozaki_update", load_library().rpcholqr_ozaki_update(
        plan.handle, _ptr(X), m, K, X.stride(0), _ptr(Y), N, Y.stride(0), _ptr(B), B.stride(0), _ptr(C),
        C.stride(0), _ptr(info), _stream(stream, X.device)))
    return C, info


def rpcholqr_ozaki_gram(plan: Plan, X, G=None, info=None, stream=None):
    """G = X^T X as a split-precision BF16 tensor-core product (SPLIT64 plan)."""
    torch = _torch()
    _mat(X, "X")
    m, n = X.shape
    if G is None:
        G = torch.empty((n, n), dtype=torch.float64, device=X.device)
    info = _info(info, X.device)
    _check("rpcholqr_ozaki_gram", load_library().rpcholqr_ozaki_gram(
        plan.handle, _ptr(X), m, n, X.stride(0), _ptr(G), _ptr(info), _stream(stream, X.device)))
    return G, info


def rpcholqr_probe_fp64_mma(device: int = 0, iters: int = 2048) -> float:
    """Measured FP64 mma.sync m16n8k16 throughput of the device, FLOP/s."""
    out = ctypes.c_double()
    _check("rpcholqr_probe_fp64_mma",
           load_library().rpcholqr_probe_fp64_mma(device, iters, ctypes.byref(out)))
    return float(out.value)


def rpcholqr_plan_enable_timing(plan: Plan, max_calls: int):
    """Record CUDA events around every phase of the next ``max_calls`` factor calls (0 disables)."""
    _check("rpcholqr_plan_enable_timing",
           load_library().rpcholqr_plan_enable_timing(plan.handle, max_calls))


def rpcholqr_plan_collect_timing(plan: Plan):
    """({phase: summed ms}, timed calls, kernel launches since the last collect)."""
    ms = (ctypes.c_float * len(PHASES))()
    calls = ctypes.c_int32()
    launches = ctypes.c_int64()
    _check("rpcholqr_plan_collect_timing", load_library().rpcholqr_plan_collect_timing(
        plan.handle, ctypes.cast(ms, ctypes.c_void_p), ctypes.byref(calls), ctypes.byref(launches)))
    return dict(zip(PHASES, [float(x) for x in ms])), int(calls.value), int(launches.value)


def rpcholqr_plan_collect_kernel_timing(plan: Plan):
    """{class: (summed ms, launches, algorithmic FP64 flops)} over the timed calls (call before
    rpcholqr_plan_collect_timing, which resets the timed calls)."""
    k = len(KERNEL_CLASSES)
    ms = (ctypes.c_float * k)()
    nl = (ctypes.c_int64 * k)()
    fl = (ctypes.c_double * k)()
    _check("rpcholqr_plan_collect_kernel_timing", load_library().rpcholqr_plan_collect_kernel_timing(
        plan.handle, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(nl, ctypes.c_void_p), ctypes.cast(fl, ctypes.c_void_p)))
    return {name: (float(ms[i]), int(nl[i]), float(fl[i])) for i, name in enumerate(KERNEL_CLASSES)}


def rpcholqr_precondition_gram_noalloc(A, Rs, A1, G, info=None, stream=None):
    """Plan-free, allocation-free fused pass (n <= 64): every buffer is the caller's.

    For callers that may not allocate device memory while running; the library's fixed device
    scratch array is used instead (see include/rpcholqr.h).  Calls must not overlap on the GPU.
    A1 (m x n), G (n x n, contiguous), Rs (n x n, contiguous) and info (int32, >= 2 entries) must
    already exist on A's device: nothing is allocated or copied here."""
    torch = _torch()
    lib = load_library()
    f = lib.rpcholqr_precondition_gram_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _mat(A, "A")
    m, n = A.shape
    _mat(Rs, "Rs")
    _mat(A1, "A1")
    _mat(G, "G")
    if tuple(A1.shape) != (m, n):
        raise ValueError(f"A1 must be {m} x {n}, got {tuple(A1.shape)}")
    if tuple(G.shape) != (n, n) or not G.is_contiguous():
        raise ValueError(f"G must be a contiguous {n} x {n} tensor")
    if tuple(Rs.shape) != (n, n) or not Rs.is_contiguous():
        raise ValueError(f"Rs must be a contiguous {n} x {n} tensor (no temporary copy is made)")
    if info is None:
        raise ValueError("info must be a device int32 tensor of >= 2 entries (nothing is allocated here)")
    if not isinstance(info, torch.Tensor) or info.dtype != torch.int32 or info.numel() < 2 \
            or not info.is_contiguous():
        raise ValueError("info must be a contiguous device int32 tensor of >= 2 entries")
    for name, t in (("Rs", Rs), ("A1", A1), ("G", G), ("info", info)):
        if t.device != A.device:
            raise ValueError(f"{name} is on {t.device}, A on {A.device}")
    with torch.cuda.device(A.device):
        _check("rpcholqr_precondition_gram_noalloc", f(
            _ptr(A), m, n, A.stride(0), _ptr(Rs), _ptr(A1), A1.stride(0), _ptr(G), _ptr(info),
            _stream(stream, A.device)))
    return A1, G, info


# ---- batches of independent matrices --------------------------------------------------------------
class Batch:
    """Owner of a C batch handle: `slots` independent plans/streams for concurrent small factorisations."""

    def __init__(self, handle, device, slots):
        self.handle = handle
        self.device = device
        self.slots = slots
        self._keep = None

    def close(self):
        if self.handle:
            load_library().rpcholqr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rpcholqr_batch_create(device: int, max_m: int, max_n: int, max_s: int, slots: int = 8,
                          mode: int = FP64) -> Batch:
    h = ctypes.c_void_p()
    _check("rpcholqr_batch_create", load_library().rpcholqr_batch_create(
        ctypes.byref(h), device, mode, max_m, max_n, max_s, slots))
    return Batch(h, device, slots)


def rpcholqr_batch_destroy(batch: Batch):
    batch.close()


def _batch_arrays(As, ss, seeds, Qs, Rs):
    count = len(As)
    P = ctypes.c_void_p * count
    arrs = {
        "A": P(*[t.data_ptr() for t in As]),
        "m": (ctypes.c_int64 * count)(*[t.shape[0] for t in As]),
        "n": (ctypes.c_int32 * count)(*[t.shape[1] for t in As]),
        "lda": (ctypes.c_int64 * count)(*[t.stride(0) for t in As]),
        "s": (ctypes.c_int32 * count)(*ss),
        "seed": (ctypes.c_uint64 * count)(*seeds),
        "Q": P(*[t.data_ptr() for t in Qs]),
        "ldq": (ctypes.c_int64 * count)(*[t.stride(0) for t in Qs]),
        "R": P(*[t.data_ptr() for t in Rs]),
    }
    args = [count] + [ctypes.cast(arrs[k], ctypes.c_void_p) for k in
                      ("A", "m", "n", "lda", "s", "seed", "Q", "ldq", "R")]
    return args, arrs


def _batch_outputs(As, Qs, Rs, info):
    torch = _torch()
    dev = As[0].device
    if Qs is None:
        Qs = [torch.empty_like(a) for a in As]
    if Rs is None:
        Rs = [torch.empty((a.shape[1], a.shape[1]), dtype=torch.float64, device=dev) for a in As]
    if info is None:
        info = torch.empty(2 * len(As), dtype=torch.int32, device=dev)
    for a in As:
        _mat(a, "A")
    return Qs, Rs, info


def rpcholqr_batch_factor(batch: Batch, As, ss, seeds, Qs=None, Rs=None, info=None, stream=None):
    """Factor the list of device matrices As (s[i] samples, seeds[i]) on the batch's slot plans; returns
    (Qs, Rs, info[2*count])."""
    Qs, Rs, info = _batch_outputs(As, Qs, Rs, info)
    args, _keep = _batch_arrays(As, ss, seeds, Qs, Rs)
    _check("rpcholqr_batch_factor", load_library().rpcholqr_batch_factor(
        batch.handle, *args, _ptr(info), _stream(stream, As[0].device)))
    return Qs, Rs, info


class BatchArrays:
    """Device-resident per-matrix arrays of a batch (pointers and shapes), as rpcholqr_factor_batched takes
    them; built once from lists of tensors and reusable across calls (and CUDA-graph replays)."""

    def __init__(self, As, ss, seeds, Qs, Rs):
        torch = _torch()
        dev = As[0].device
        i64 = torch.int64

        def arr(vals, dtype):
            return torch.tensor(vals, dtype=dtype).to(dev)

        def u64(v):   # uint64 bit patterns carried in int64
            v = int(v) & 0xFFFFFFFFFFFFFFFF
            return v - (1 << 64) if v >= (1 << 63) else v

        self.count = len(As)
        self.A = arr([t.data_ptr() for t in As], i64)
        self.m = arr([t.shape[0] for t in As], i64)
        self.n = arr([t.shape[1] for t in As], torch.int32)
        self.lda = arr([t.stride(0) for t in As], i64)
        self.s = arr(list(ss), torch.int32)
        self.seed = arr([u64(x) for x in seeds], i64)
        self.Q = arr([t.data_ptr() for t in Qs], i64)
        self.ldq = arr([t.stride(0) for t in Qs], i64)
        self.R = arr([t.data_ptr() for t in Rs], i64)
        self.keep = (As, Qs, Rs)

    def args(self):
        return [self.count] + [_ptr(getattr(self, k)) for k in ("A", "m", "n", "lda", "s", "seed", "Q", "ldq", "R")]


def rpcholqr_factor_batched(plan: Plan, As, ss, seeds, Qs=None, Rs=None, info=None, stream=None, arrays=None):
    """All matrices of the list As in one persistent kernel launch (FP64 plan, n <= 128); returns
    (Qs, Rs, info[2*count], arrays).  `arrays` (a BatchArrays of the same tensors) may be passed to reuse
    the device-resident pointer/shape arrays."""
    Qs, Rs, info = _batch_outputs(As, Qs, Rs, info)
    if arrays is None:
        arrays = BatchArrays(As, ss, seeds, Qs, Rs)
    _check("rpcholqr_factor_batched", load_library().rpcholqr_factor_batched(
        plan.handle, *arrays.args(), _ptr(info), _stream(stream, As[0].device)))
    return Qs, Rs, info, arrays


def rpcholqr_batch_capture(batch: Batch, As, ss, seeds, Qs=None, Rs=None, info=None, stream=None):
    """Capture the batched factorisation into a CUDA graph (replay with rpcholqr_batch_replay)."""
    Qs, Rs, info = _batch_outputs(As, Qs, Rs, info)
    args, keep = _batch_arrays(As, ss, seeds, Qs, Rs)
    _check("rpcholqr_batch_capture", load_library().rpcholqr_batch_capture(
        batch.handle, *args, _ptr(info), _stream(stream, As[0].device)))
    batch._keep = (As, Qs, Rs, info, keep)
    return Qs, Rs, info


def rpcholqr_batch_replay(batch: Batch, stream=None):
    torch = _torch()
    _check("rpcholqr_batch_replay", load_library().rpcholqr_batch_replay(
        batch.handle, _stream(stream, torch.device("cuda", batch.device))))


def rpcholqr_batch_autotune(batch: Batch, As, ss, seeds, Qs=None, Rs=None, info=None, reps: int = 2,
                            stream=None):
    """Pick the fastest number of concurrent slots for this batch; returns (slots, ms per batch)."""
    Qs, Rs, info = _batch_outputs(As, Qs, Rs, info)
    args, _keep = _batch_arrays(As, ss, seeds, Qs, Rs)
    best = ctypes.c_int32()
    ms = ctypes.c_float()
    _check("rpcholqr_batch_autotune", load_library().rpcholqr_batch_autotune(
        batch.handle, *args, _ptr(info), reps, ctypes.byref(best), ctypes.byref(ms),
        _stream(stream, As[0].device)))
    return int(best.value), float(ms.value)
