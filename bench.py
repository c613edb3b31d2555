#!/usr/bin/env python
"""Throughput of rpCholesky-QR (Garrison & Ipsen, arXiv 2406.11751, Algorithm alg_2) on GB300.

One step = one full rpcholqr_factor call (sample + Householder R_s + preconditioning pass + Gram +
Cholesky + second pass + R recovery) on an m x n FP64 matrix resident in HBM.

Default workload (--config 5, the largest single-GPU workload): m = 2^23, n = 512, s = 3n = 1536,
A = U diag(sigma) V^T with sigma log-spaced from 1 to 1e-18 (numerically singular), U, V Haar;
SPLIT64 mode, with the plain FP64 mode timed beside it ("other_mode") and the m = 2^20, n = 128,
kappa = 1e8 workload (--config 2) reported under "config2", with its kappa sweep (kappa 1 to 1e16,
s = 3n and 10n, both modes, Cholesky-QR2 beside each kappa; --preset kappa-sweep runs config 2 with the
sweep alone).  A (34.4 GB) is larger than L2, so
consecutive steps do not reuse cached inputs.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 1|2|3|5]

--impl reference times the FP64 CPU oracle (the only "reference" this project has: the paper
ships no code) on the host cores, each step one oracle call on a bounded row sample of the same
workload; its ms_per_step is that measured call, its value the per-matrix rate extrapolated from two
sample sizes (the oracle's cost is a fixed part plus a part linear in m).
Under torchrun (N > 1) every rank factors its own matrix (independent problems, weak scaling,
no collective on the data path); rank 0 prints the aggregate over max-over-ranks time.
--profile-window brackets the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TS-QR matrices/s & effective TFLOP/s at ||Q^T Q - I||_2 <= 1e-13; % of roofline"


# The workloads (sigma log-spaced from 1 to 1/kappa, s = 3n): 1 = 10,000 x 50, kappa 1e8; 2 = 2^20 x 128,
# kappa 1e8; 3 = 2^22 x 256, kappa 1e12 (1e5 for the FP32 variant); 5 = 2^23 x 512, sigma to 1e-18.
# (4 is the heterogeneous batch: --workload batch.)
CONFIGS = {1: (10000, 50, 1e8), 2: (1 << 20, 128, 1e8), 3: (1 << 22, 256, 1e12), 5: (1 << 23, 512, 1e18)}
PRESETS = {"small": 1, "headline": 2, "precision": 3, "large": 5, "kappa-sweep": 2}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, choices=sorted(CONFIGS), default=5,
                    help="workload: 1 = 10,000 x 50; 2 = 2^20 x 128; 3 = 2^22 x 256; 5 = 2^23 x 512 (default)")
    ap.add_argument("--preset", choices=sorted(PRESETS), default=None,
                    help="alias of --config: small 1, headline 2, precision 3, large 5; kappa-sweep: config 2 "
                         "plus its kappa sweep (kappa 1..1e16, s 3n and 10n, both modes, Cholesky-QR2 beside)")
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--s", type=int, default=None, help="sampled rows (default 3n)")
    ap.add_argument("--kappa", type=float, default=None)
    ap.add_argument("--seed", type=int, default=20240617)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="host-buffer end-to-end steps (default 3, 2 above 2^21 rows)")
    ap.add_argument("--other-steps", type=int, default=None,
                    help="timed steps of the other mode (default: --steps up to 2^21 x 128 elements, else 2)")
    ap.add_argument("--cpu-sample-rows", type=int, default=None,
                    help="rows of the oracle's bounded sample (default 2^17 at n = 128, scaled by (128/n)^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inputs", choices=["gpu", "cpu"], default="gpu",
                    help="draw A with torch on the GPU (fast) or with the numpy recipe on the host")
    ap.add_argument("--no-metrics", action="store_true", help="skip the orthogonality/residual check")
    ap.add_argument("--mode", choices=["fp64", "split", "fp32"], default="split",
                    help="split (default): FP64-accurate Ozaki-split BF16 tensor-core products for the "
                         "well-conditioned steps; fp64: every step in FP64; fp32: float data, FP32 "
                         "passes (FP64 sketch QR and Cholesky)")
    ap.add_argument("--workload", choices=["single", "batch"], default="single",
                    help="single: one m x n matrix per step; batch: the 512-matrix heterogeneous batch "
                         "(m log-uniform in [4096, 2^20], n in {8..128}, s=3n, kappa log-uniform in "
                         "[1, 1e14]) per step, one CUDA-graph replay")
    ap.add_argument("--smoothing", choices=["none", "wht", "dct"], default="none",
                    help="sample the smoothed F A (Algorithm alg_2 with F = F_T D): Walsh-Hadamard or cosine F_T")
    ap.add_argument("--count", type=int, default=512, help="matrices in the batch workload")
    ap.add_argument("--slots", type=int, default=16, help="concurrent slots the batch autotuner may use")
    ap.add_argument("--no-compare", action="store_true",
                    help="do not also time the other mode (reported as 'other_mode')")
    ap.add_argument("--no-config2", action="store_true",
                    help="with --config 5: do not also time the 2^20 x 128 workload ('config2') nor the batch")
    ap.add_argument("--no-config4", action="store_true",
                    help="with --config 5: do not also time the 512-matrix batch ('config4')")
    ap.add_argument("--sharded", action="store_true",
                    help="one m x n matrix split by rows over the N processes (row-sharded factorisation: "
                         "FP64 steps, the sample and the Gram partials exchanged over NCCL; strong scaling)")
    ap.add_argument("--image-rows", type=int, default=0,
                    help="SPLIT64 above 128 columns: stage-image rows kept at a time (plan option "
                         "RPCHOLQR_OPT_IMAGE_ROWS; 0 = automatic: every row when they fit a quarter of the device)")
    ap.add_argument("--profile-window", action="store_true",
                    help="cudaProfilerStart/Stop around the timed steps of the main mode only")
    args = ap.parse_args(argv)
    args.kappa_sweep = args.preset == "kappa-sweep"
    if args.preset:
        args.config = PRESETS[args.preset]
    m, n, kappa = CONFIGS[args.config]
    if args.config == 3 and args.mode == "fp32":
        kappa = 1e5     # the single-precision variant of that workload
    args.m = args.m or m
    args.n = args.n or n
    args.kappa = args.kappa or kappa
    if args.e2e_steps is None:
        args.e2e_steps = 3 if args.m <= (1 << 21) else 2
    if args.other_steps is None:
        args.other_steps = args.steps if args.m * args.n <= (1 << 21) * 128 else 2
    if args.cpu_sample_rows is None:
        # about the same oracle work (rows x n^2) at every width, and at least twice the sample size
        args.cpu_sample_rows = max(4096, min(args.m, (1 << 17) * 128 * 128 // (args.n * args.n)))
        args.cpu_sample_rows = min(args.m, max(args.cpu_sample_rows, 2 * (args.s or 3 * args.n)))
    return args


def alg_flops(m, n, s):
    """3mn^2 (two row-solve passes + Gram) + 2sn^2 (sketch QR) + 2n^3/3 (Cholesky + R product)."""
    return 3.0 * m * n * n + 2.0 * s * n * n + 2.0 * n ** 3 / 3.0


# ---- clocks sampled during the timed region --------------------------------------------------------
class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def summary(self):
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        if not self.lines:
            return None
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- distributed helpers (torchrun) -----------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def max_over_ranks(value, dist, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---- metrics on the device (after timing) -----------------------------------------------------------
def gpu_metrics(A, Q, R, rows=1 << 18):
    """||Q^T Q - I||_2 and ||A - QR||_2 / ||A||_2 in FP64 from n x n Gram matrices of row chunks (each
    chunk's Gram summed over 4096-row blocks, chunks added in order); no m x n temporaries."""
    import torch
    m, n = Q.shape
    blk = 4096

    def gram(X):
        k = X.shape[0]
        full = (k // blk) * blk
        G = torch.zeros((n, n), dtype=torch.float64, device=X.device)
        if full:
            parts = torch.bmm(X[:full].view(-1, blk, n).transpose(1, 2), X[:full].view(-1, blk, n))
            while parts.shape[0] > 1:
                h = parts.shape[0] // 2
                parts = torch.cat([parts[:h] + parts[h:2 * h], parts[2 * h:]], 0)
            G += parts[0]
        if full < k:
            G += X[full:].T @ X[full:]
        return G

    QQ = torch.zeros((n, n), dtype=torch.float64, device=Q.device)
    DD = torch.zeros_like(QQ)
    AA = torch.zeros_like(QQ)
    for i in range(0, m, rows):
        q, a = Q[i:i + rows], A[i:i + rows]
        QQ += gram(q)
        DD += gram(a - q @ R)
        AA += gram(a)
    E = QQ - torch.eye(n, dtype=torch.float64, device=Q.device)
    orth = float(torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max())
    nd = float(torch.linalg.eigvalsh(DD).abs().max().sqrt())
    na = float(torch.linalg.eigvalsh(AA).abs().max().sqrt())
    return orth, nd / na


def traffic_from_profiles(cls, n, src_file, m, launches_per_call):
    """DRAM bytes per launch of a kernel class from profiles/traffic.txt, when the class's source file is
    unchanged since the capture.  A line holds one call's total for the class at `measured_m` rows and width
    n; the streaming kernels' traffic is proportional to the rows, so the total is scaled to m and divided
    by the launches the class makes in one call at m."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src_file, "rb").read()).hexdigest()[:16]
    for line in open(path):
        if line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("class") == cls and f.get("n") == str(n) and f.get("src_sha") == sha:
            try:
                per_call = float(f["dram_bytes_per_call"]) * m / float(f["measured_m"])
            except (KeyError, ValueError):
                return None
            return per_call / max(launches_per_call, 1)
    return None


# ---- the oracle on the host cores --------------------------------------------------------------------
def oracle_calls(m, n, s, kappa, seed, rows, reps, warm=1):
    """Times `reps` oracle rpCholesky-QR calls on the first `rows` rows of the workload (same n, s,
    kappa), after `warm` untimed calls and the best of two calls on rows/2 rows: (per-call seconds of
    the `reps` calls, half-sample seconds, rows, half rows, threads used).  The two sizes separate the
    oracle's fixed cost (sample, Householder QR, Cholesky) from its per-row cost, so the full-m time
    is extrapolated as t + (m - rows) * per_row."""
    import inputs
    import oracle
    oracle.build()
    rows = min(rows, m)
    half = max(min(s, rows), rows // 2)
    A = inputs.usv(rows, n, kappa, seed)
    Ah = np_ascontig(A[:half])

    def call(X, k):
        t0 = time.perf_counter()
        o = oracle.rpcholqr(X, min(s, X.shape[0]), 1 + k)
        dt = time.perf_counter() - t0
        if o["status"] != 0:
            raise RuntimeError(f"oracle status {o['status']}")
        return dt

    for w in range(max(warm, 1)):
        call(A, w)
    t_half = min(call(Ah, 0), call(Ah, 1))
    times = [call(A, r) for r in range(reps)]
    return times, t_half, rows, half, oracle.num_threads()


def np_ascontig(a):
    import numpy as np
    return np.ascontiguousarray(a)


def extrapolate_full(t_rows, t_half, rows, half, m):
    """Seconds for the full m from calls on `rows` and `half` rows (cost = fixed + per_row * rows)."""
    if rows >= m:
        return t_rows
    per_row = max(t_rows - t_half, 0.0) / max(rows - half, 1) if rows > half else t_rows / rows
    if per_row <= 0.0:
        per_row = t_rows / rows
    return t_rows + (m - rows) * per_row


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    m, n = args.m, args.n
    s = args.s or 3 * n
    timed, t_half, rows, half, cores = oracle_calls(m, n, s, args.kappa, args.seed, args.cpu_sample_rows,
                                                     args.steps, warm=args.warmup)
    per_step = sum(timed) / len(timed)
    full = extrapolate_full(per_step, t_half, rows, half, m)
    value = 1.0 / full
    sample = (f"each step one oracle rpCholesky-QR call on the first {rows} of {m} rows (same n, s, kappa; "
              f"{per_step * 1e3:.1f} ms measured per step); value = per-matrix rate extrapolated to the full m "
              f"from that call and one on {half} rows ({t_half * 1e3:.1f} ms): {full * 1e3:.1f} ms per matrix")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matrices/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rpCholesky-QR m={m} n={n} s={s} kappa={args.kappa:g}", "m": m, "n": n,
                   "s": s, "kappa": args.kappa},
        "value_basis": "extrapolated" if rows < m else "measured",
        "extrapolated_ms_per_matrix": full * 1e3,
        "sample_rows": rows,
        "effective_tflops": alg_flops(m, n, s) * value / 1e12,
        "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---- our CUDA path -------------------------------------------------------------------------------------
MODES = ("fp64", "split", "fp32")


def preload_torch_linalg():
    """Load torch's CUDA linear-algebra library by full path before torch.linalg first needs it (the
    input generator's QR): under ncu's injection torch's own lazy dlopen of it by name fails."""
    import ctypes
    import torch
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def timed_factor(rq, torch, local, dev, dist, m, n, s, mode, A, Q, R, info, stream, K, W, smoothing="none",
                 clocks=False, profile=False, A32=None, Q32=None, R32=None, image_rows=0):
    """W warm-up + K timed factor calls on a fresh plan of `mode` (CUDA events on the launching stream,
    barrier + synchronize on both sides): (ms over the K steps, phases, calls, launches, plan, clocks)."""
    modes = {"fp64": rq.FP64, "split": rq.SPLIT64, "fp32": rq.FP32}

    def factor(plan, seed):
        if mode == "fp32":
            rq.rpcholqr_factor_f32(plan, A32, s, seed, Q=Q32, R=R32, info=info, stream=stream)
        else:
            rq.rpcholqr_factor(plan, A, s, seed, Q=Q, R=R, info=info, stream=stream)

    plan = rq.rpcholqr_plan_create(local, m, n, s, mode=modes[mode])
    if image_rows and mode == "split" and n > 128:
        rq.rpcholqr_plan_set_option(plan, rq.OPT_IMAGE_ROWS, image_rows)
    if smoothing != "none":
        rq.rpcholqr_plan_set_smoothing(plan, rq.SMOOTH_WHT if smoothing == "wht" else rq.SMOOTH_DCT)
    for w in range(W):
        factor(plan, 1 + w)
    torch.cuda.synchronize(dev)
    st0 = info.cpu().tolist()
    if st0[0] != 0:
        raise RuntimeError(f"{mode} warm-up status {rq.rpcholqr_status_string(st0[0])}")
    rq.rpcholqr_plan_collect_timing(plan)          # reset counters
    rq.rpcholqr_plan_enable_timing(plan, K)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with (ClockSampler(local) if clocks else _NoClock()) as clk:
        barrier(dist)
        torch.cuda.synchronize(dev)
        if profile:
            torch.cuda.profiler.start()
        e0.record(stream)
        for k in range(K):
            factor(plan, 1 + k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if profile:
            torch.cuda.profiler.stop()
        barrier(dist)
    kt = rq.rpcholqr_plan_collect_kernel_timing(plan)
    ph, calls, launches = rq.rpcholqr_plan_collect_timing(plan)
    rq.rpcholqr_plan_enable_timing(plan, 0)
    ph["kernels"] = kt
    return max_over_ranks(e0.elapsed_time(e1), dist, dev), ph, calls, launches, plan, clk


def phases_per_step(ph, calls):
    return {k: v / max(calls, 1) for k, v in ph.items() if k != "kernels"}


def kernels_per_step(ph, calls):
    """{class: {ms, launches, fp64_gflop}} per step, for the classes that ran."""
    c = max(calls, 1)
    return {k: {"ms": ms / c, "launches": nl / c, "fp64_gflop": fl / c / 1e9}
            for k, (ms, nl, fl) in ph.get("kernels", {}).items() if nl > 0}


# Each FP64-accurate split product runs 36 BF16 slice products (eight 7-bit slices per operand, the pairs
# with a + b <= 9); the tensor roofline of a split kernel counts those BF16 flops.
SLICE_PRODUCTS = 36
SPLIT_CLASSES = ("split_update", "split_gemm_sub", "split_gemm", "split_gram")
KERNEL_NAMES = {
    "rowpass": "k_rowpass (FP64 row solves: mma.sync m16n8k16 + DFMA)",
    "split_update": "oz::k_ozaki_update (split C = B - X Y, K <= 32)",
    "split_gemm_sub": "oz::k_ozaki_gemm_db<SUB> (n > 128; k_ozaki_gemm_ws<.,SUB> up to 128) (split C = B - X Y, "
                      "wide pass-1 block updates)",
    "split_gemm": "oz::k_ozaki_gemm_db (n > 128; k_ozaki_gemm_ws up to 128) (split Q = A1 R1^-1)",
    "split_gram": "oz::k_ozaki_gram (split G1 = A1^T A1)",
    "fp64_gemm": "k_gemm_sub_fp64 (FP64 block updates)",
    "fp64_syrk": "k_syrk_fp64 (FP64 Gram)",
    "sketch_qr": "k_hh_cluster (Householder QR of the sample)",
    "cholesky": "k_cholesky (G1 = R1^T R1)",
}


CLASS_SOURCE = {"rowpass": "rowpass.cuh", "split_update": "ozaki.cu", "split_gemm_sub": "ozaki.cu",
                "split_gemm": "ozaki.cu", "split_gram": "ozaki.cu", "fp64_gemm": "blocked.cu",
                "fp64_syrk": "blocked.cu", "sketch_qr": "smallfactor.cuh", "cholesky": "smallfactor.cuh"}


def class_bytes(cls, mode, m, n):
    """Algorithmic DRAM bytes per step of a kernel class: what its launches must read and write at least
    (FP64 values, each once per launch that needs it)."""
    nb = (n + 63) // 64
    if cls == "rowpass":
        if mode == "split":
            return 16.0 * m * n                     # pass-1 diagonal blocks: each column read and written once
        return 32.0 * m * n                         # pass 1 and pass 2, each column read and written once
    if cls == "split_gemm":
        return 16.0 * m * n                         # read A1, write Q
    if cls == "split_gram":
        return 8.0 * m * n                          # read A1
    if cls in ("split_gemm_sub", "fp64_gemm"):     # left-looking 64-column blocks: read A1[:, <J], B, write C
        return sum(8.0 * m * (64 * J + 2 * 64) for J in range(1, nb))
    if cls == "split_update":
        return 8.0 * m * 3 * n                      # X, B, C columns of the updates, about n each
    if cls == "fp64_syrk":
        return 8.0 * m * n
    return 0.0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def kernel_rooflines(phases, calls, fp64_peak_tflops):
    """Roofline entry per kernel class from the per-launch CUDA events of the timed steps: FP64 classes
    against the FP64 pipe (in-run probe), split classes against the BF16 tensor pipe (sustained cuBLAS
    figure of MEASURED_PEAKS.json: these kernels run inside a seconds-long step) counting the 36 slice
    products of each FP64-accurate product."""
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    out = {}
    for k, v in kernels_per_step(phases, calls).items():
        if v["ms"] <= 0:
            continue
        fp64_tf = v["fp64_gflop"] / v["ms"]          # GFLOP / ms = TFLOP/s
        if k in SPLIT_CLASSES:
            achieved = SLICE_PRODUCTS * fp64_tf
            e = {"kernel": KERNEL_NAMES[k], "bound": "tensor", "achieved": achieved, "peak": bf16,
                 "unit": "TFLOP/s", "frac": achieved / bf16 if bf16 else None, "fp64_equivalent_tflops": fp64_tf,
                 "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured); achieved counts "
                                "36 BF16 slice products per FP64 product"}
        else:
            e = {"kernel": KERNEL_NAMES[k], "bound": "alu", "achieved": fp64_tf, "peak": fp64_peak_tflops,
                 "unit": "TFLOP/s", "frac": fp64_tf / fp64_peak_tflops,
                 "peak_source": "FP64 pipe: in-run mma.sync m16n8k16 probe (MEASURED_PEAKS.json has no FP64 "
                                "figure; unit count x clock: 152 SM x 4 x 32 lanes / 64 cycles x 2 flop x "
                                "2.07 GHz = 1.26 TFLOP/s)"}
        e.update({"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                  "ms_per_launch": v["ms"] / v["launches"], "algorithmic_fp64_flops_per_launch":
                  v["fp64_gflop"] * 1e9 / v["launches"]})
        out[k] = e
    return out


def cpu_baseline_entry(m, n, s, kappa, seed, rows):
    times, t_half, rows, half, cores = oracle_calls(m, n, s, kappa, seed, rows, 3)
    full = extrapolate_full(min(times), t_half, rows, half, m)
    return {"value": 1.0 / full, "unit": "matrices/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle rpCholesky-QR on the first {rows} of {m} rows (numpy-generated, same n, s, "
                      f"kappa), best of 3 ({min(times) * 1e3:.1f} ms), and one call on {half} rows "
                      f"({t_half * 1e3:.1f} ms); full-m time extrapolated from the two: {full * 1e3:.1f} ms"}


KAPPA_SWEEP = (1.0, 1e4, 1e8, 1e12, 1e16)


def timed_cholqr2(rq, torch, local, dev, dist, A, Q, R, info, stream, K, W):
    """Cholesky-QR2 (the paper's breakdown reference) on the FP64 plan: (ms over K calls or None, status
    of the first call).  A call that breaks down (G not numerically SPD) is reported, not timed."""
    m, n = A.shape
    plan = rq.rpcholqr_plan_create(local, m, n, 3 * n, mode=rq.FP64)
    try:
        rq.rpcholqr_cholqr2(plan, A, Q=Q, R=R, info=info, stream=stream)
        torch.cuda.synchronize(dev)
        st = info.cpu().tolist()[0]
        if st != 0:
            return None, st
        for _ in range(W):
            rq.rpcholqr_cholqr2(plan, A, Q=Q, R=R, info=info, stream=stream)
        barrier(dist)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            rq.rpcholqr_cholqr2(plan, A, Q=Q, R=R, info=info, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        barrier(dist)
        return ms, info.cpu().tolist()[0]
    finally:
        plan.close()


def run_config2(args, rq, torch, local, dev, dist, stream, ws, sweep=True):
    """The 2^20 x 128 workload (sigma log-spaced, s = 3n) in SPLIT64 and FP64.  "split"/"fp64" are the
    kappa = 1e8, s = 3n figures; with `sweep`, "kappa_sweep" repeats both modes for kappa in
    {1, 1e4, 1e8, 1e12, 1e16} and s in {3n, 10n}, each entry with matrices/s, status, orthogonality and
    residual, and Cholesky-QR2 on the same A beside each kappa (its breakdown is the reference point)."""
    import inputs
    m, n, kappa0 = CONFIGS[2]
    Q = torch.empty((m, n), dtype=torch.float64, device=dev)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    info = torch.empty(2, dtype=torch.int32, device=dev)
    out = {"workload": f"rpCholesky-QR m={m} n={n} s={3 * n} kappa={kappa0:g}", "m": m, "n": n, "s": 3 * n,
           "kappa": kappa0}
    entries, cq2 = [], []
    for kappa in (KAPPA_SWEEP if sweep else (kappa0,)):
        A = inputs.usv_torch(m, n, kappa, args.seed + 7, dev)
        for s in ((3 * n, 10 * n) if sweep else (3 * n,)):
            for mode in ("split", "fp64"):
                ms, ph, calls, _, plan, _ = timed_factor(rq, torch, local, dev, dist, m, n, s, mode, A, Q, R, info,
                                                         stream, args.steps, args.warmup)
                plan.close()
                st = info.cpu().tolist()
                orth, res = (None, None) if args.no_metrics else gpu_metrics(A, Q, R)
                e = {"kappa": kappa, "s": s, "mode": mode, "value": ws * args.steps / (ms / 1e3),
                     "unit": "matrices/s", "ms_per_step": ms / args.steps, "status": st[0], "orth": orth,
                     "residual": res, "effective_tflops": alg_flops(m, n, s) * args.steps / (ms / 1e3) / 1e12}
                entries.append(e)
                if kappa == kappa0 and s == 3 * n:
                    out[mode] = dict(e, phases_ms_per_step=phases_per_step(ph, calls))
        if sweep:
            ms, st = timed_cholqr2(rq, torch, local, dev, dist, A, Q, R, info, stream, args.steps, args.warmup)
            orth, res = (None, None) if (args.no_metrics or st != 0) else gpu_metrics(A, Q, R)
            cq2.append({"kappa": kappa, "status": rq.rpcholqr_status_string(st),
                        "value": None if ms is None else ws * args.steps / (ms / 1e3), "unit": "matrices/s",
                        "ms_per_step": None if ms is None else ms / args.steps, "orth": orth, "residual": res})
        del A
        torch.cuda.empty_cache()
    out["split_over_fp64"] = out["split"]["value"] / out["fp64"]["value"]
    if sweep:
        out["kappa_sweep"] = entries
        out["cholqr2"] = cq2
    del Q
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local):
    import torch

    import inputs
    import paper_2406_11751_gb300 as rq

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(ws, "nccl")
    rq.build()
    preload_torch_linalg()
    m, n = args.m, args.n
    s = args.s or 3 * n
    K, W = args.steps, args.warmup

    if args.inputs == "gpu":
        A = inputs.usv_torch(m, n, args.kappa, args.seed + rank, dev)
    else:
        A = torch.from_numpy(inputs.usv(m, n, args.kappa, args.seed + rank)).to(dev)
    Q = torch.empty_like(A)
    R = torch.empty((n, n), dtype=torch.float64, device=dev)
    info = torch.empty(2, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.empty_cache()    # the generator's temporaries back to the device before the plans allocate
    fp64_peak = rq.rpcholqr_probe_fp64_mma(local, 4096)
    A32 = Q32 = R32 = None
    if args.mode == "fp32":
        A32 = A.float()
        Q32 = torch.empty_like(A32)
        R32 = torch.empty((n, n), dtype=torch.float32, device=dev)

    def run(mode, steps, warm, clocks=False, profile=False):
        return timed_factor(rq, torch, local, dev, dist, m, n, s, mode, A, Q, R, info, stream, steps, warm,
                            smoothing=args.smoothing, clocks=clocks, profile=profile, A32=A32, Q32=Q32, R32=R32,
                            image_rows=args.image_rows)

    other = None
    if not args.no_compare:
        omode = {"split": "fp64", "fp64": "split", "fp32": "split"}[args.mode]
        ok = args.other_steps
        ow = W if ok == K else 1
        o_ms, o_ph, o_calls, _, o_plan, _ = run(omode, ok, ow)
        o_plan.close()
        other = {"mode": omode, "value": ws * ok / (o_ms / 1e3), "ms_per_step": o_ms / ok, "steps": ok,
                 "warmup": ow, "phases_ms_per_step": phases_per_step(o_ph, o_calls)}
    t_ms_max, phases, calls, launches, plan, clk = run(args.mode, K, W, clocks=True, profile=args.profile_window)
    st = info.cpu().tolist()
    image_rows = None
    if args.mode == "split" and n > 128:
        image_rows = rq.rpcholqr_plan_get_option(plan, rq.OPT_IMAGE_ROWS)
    if args.no_metrics:
        orth, res = None, None
    elif args.mode == "fp32":
        orth, res = gpu_metrics(A32.double(), Q32.double(), R32.double())
    else:
        orth, res = gpu_metrics(A, Q, R)

    # end to end through the host-buffer C-ABI call (H2D of A, D2H of Q, R, info inside the region)
    e2e = None
    if args.e2e_steps > 0 and args.mode == "fp32":
        # through the public Python API: pinned host A -> device, factor, Q, R, info -> pinned host
        Ah = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
        Ah.copy_(A32)
        Qh = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
        Rh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        ih = torch.empty(2, dtype=torch.int32, pin_memory=True)
        Ad = torch.empty_like(A32)
        barrier(dist)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            Ad.copy_(Ah, non_blocking=True)
            rq.rpcholqr_factor_f32(plan, Ad, s, 1 + k, Q=Q32, R=R32, info=info, stream=stream)
            Qh.copy_(Q32, non_blocking=True)
            Rh.copy_(R32, non_blocking=True)
            ih.copy_(info, non_blocking=True)
            torch.cuda.synchronize(dev)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        barrier(dist)
        e2e = {"value": ws * args.e2e_steps / e2e_s, "unit": "matrices/s", "steps": args.e2e_steps,
               "h2d_bytes_per_step": 4 * m * n, "d2h_bytes_per_step": 4 * m * n + 4 * n * n + 8}
        del Ah, Qh, Ad
    elif args.e2e_steps > 0:
        Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        Qh = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        rq.rpcholqr_factor_host(plan, Ah, s, 1, Q=Qh, R=Rh, stream=stream)   # allocates staging
        barrier(dist)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            rq.rpcholqr_factor_host(plan, Ah, s, 1 + k, Q=Qh, R=Rh, stream=stream)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        barrier(dist)
        e2e = {"value": ws * args.e2e_steps / e2e_s, "unit": "matrices/s", "steps": args.e2e_steps,
               "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * m * n + 8 * n * n + 8}
        del Ah, Qh

    config2 = config4 = None
    if args.config == 5 and not args.no_config2 and not args.profile_window and args.mode != "fp32" \
            and args.smoothing == "none":
        plan.close()
        plan = None
        del A, Q
        torch.cuda.empty_cache()
        config2 = run_config2(args, rq, torch, local, dev, dist, stream, ws)
        if not args.no_config4:
            config4 = run_config4(args, rq, torch, local, dev, dist, ws)
    elif args.kappa_sweep:
        plan.close()
        plan = None
        del A, Q
        torch.cuda.empty_cache()
        config2 = run_config2(args, rq, torch, local, dev, dist, stream, ws)

    if rank != 0:
        if plan is not None:
            plan.close()
        return 0

    N = ws
    value = N * K / (t_ms_max / 1e3)
    flops = alg_flops(m, n, s)
    np_ = (n + 15) // 16 * 16
    src = os.path.join(ROOT, "paper_2406_11751_gb300", "csrc", "rowpass.cu")
    c = max(calls, 1)
    fp32_peak = 152 * 128 * 2 * 2.07e9   # FP32 FMA lanes x 2 flop x max SM clock
    if args.mode == "fp32":
        kname = "k_rowsolve_f32 (FP32 pass 1: A1 = A Rs^-1, one row per thread)"
        launches_per_call = 1
        k_ms = phases["pass1"] / c
        k_flops = float(m) * n * n          # n^2/2 FMAs per row
        k_bytes = 8.0 * m * n               # read A, write A1 (float)
        traffic = None
    rooflines = None
    if args.mode == "fp32":
        achieved = k_flops / (k_ms / 1e3) / 1e12
        peak = fp32_peak / 1e12
        roofline = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "algorithmic_flops": k_flops,
                    "algorithmic_bytes": k_bytes, "ms_per_launch": k_ms, "launches_per_step": launches_per_call,
                    "peak_source": "FP32 FMA pipe from unit counts and clock: 152 SM x 128 lanes x 2 flop x "
                                   "2.07 GHz = 80.5 TFLOP/s (MEASURED_PEAKS.json has no FP32 figure)"}
    else:
        # every kernel class from its own per-launch CUDA events inside the timed steps; the dominant one
        # (the most time per step) is the line's roofline
        rooflines = kernel_rooflines(phases, calls, fp64_peak / 1e12)
        dom = max(rooflines, key=lambda k: rooflines[k]["ms_per_step"])
        roofline = dict(rooflines[dom])
        roofline["class"] = dom
        roofline["algorithmic_bytes_per_launch"] = class_bytes(dom, args.mode, m, n) / roofline["launches_per_step"]
        roofline["traffic"] = traffic_from_profiles(dom, n, os.path.join(
            ROOT, "paper_2406_11751_gb300", "csrc", CLASS_SOURCE[dom]), m, roofline["launches_per_step"])
        for cls, r in rooflines.items():
            r["traffic"] = traffic_from_profiles(cls, n, os.path.join(
                ROOT, "paper_2406_11751_gb300", "csrc", CLASS_SOURCE[cls]), m, r["launches_per_step"])

    cpu = None
    if not args.no_cpu_baseline and N == 1:
        cpu = cpu_baseline_entry(m, n, s, args.kappa, args.seed, max(args.cpu_sample_rows, 4 * s))

    out = {
        "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": N, "steps": K, "warmup": W,
        "ms_per_step": t_ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "split": "f64+bf16", "fp32": "f32+f64"}[args.mode],
        "data": "synthetic (A = U diag(sigma) V^T, Haar U/V from torch, sigma log-spaced)",
        "config": {"workload": f"rpCholesky-QR {args.mode.upper()} m={m} n={n} s={s} kappa={args.kappa:g}"
                               + ("" if args.smoothing == "none" else f" smoothing={args.smoothing.upper()}"), "m": m,
                   "n": n, "s": s, "kappa": args.kappa, "mode": args.mode, "smoothing": args.smoothing,
                   "l2": f"inputs larger than L2 (A = {8 * m * n / 1e9:.2f} GB > 129 MB), no flush"},
        "effective_tflops": flops * value / 1e12,
        "orth": orth, "residual": res, "gate_orth_le_1e-13": None if orth is None else bool(orth <= 1e-13),
        "gate_orth_le_1e-5": None if orth is None else bool(orth <= 1e-5), "status": st[0],
        "phases_ms_per_step": phases_per_step(phases, calls),
        "kernels_per_step": kernels_per_step(phases, calls),
        "roofline": roofline,
        "rooflines": rooflines,
        "other_mode": other,
        "config2": config2,
        "config4": config4,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "plan": {"image_rows": image_rows},
    }
    print(json.dumps(out), flush=True)
    if plan is not None:
        plan.close()
    return 0


def run_sharded(args, ws, rank, local):
    """One global m x n matrix per step, its rows split over the N processes (contiguous blocks): the
    row-sharded factorisation of the library (local FP64 passes, the s x n sample and the n x n Gram
    partials exchanged over NCCL).  value = matrices/s of the whole job; scaling strong."""
    import torch

    import inputs
    import paper_2406_11751_gb300 as rq
    from paper_2406_11751_gb300 import sharded as sh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(ws, "nccl")
    rq.build()
    preload_torch_linalg()
    m, n = args.m, args.n
    s = args.s or 3 * n
    K, W = args.steps, args.warmup
    off, ml = sh.split_rows(m, ws, rank)
    A = inputs.usv_torch(m, n, args.kappa, args.seed, dev)    # the same global matrix on every process
    A_local = A[off:off + ml].contiguous()
    del A
    torch.cuda.empty_cache()
    plan = rq.rpcholqr_plan_create(local, max(ml, s), n, s)
    steps = sh.CudaSteps(plan)
    comm = sh.TorchDistComm() if ws > 1 else sh.SingleComm()
    stream = torch.cuda.current_stream(dev)
    for w in range(W):
        _, _, st = sh.factor_row_sharded(steps, comm, A_local, off, m, s, 1 + w)
        if st != 0:
            raise RuntimeError(f"sharded warm-up status {rq.rpcholqr_status_string(st)}")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(dist)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for k in range(K):
            Q_local, R, st = sh.factor_row_sharded(steps, comm, A_local, off, m, s, 1 + k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    t_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    plan.close()
    if rank != 0:
        return 0
    value = K / (t_ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (A = U diag(sigma) V^T, Haar U/V from torch, sigma log-spaced)",
        "config": {"workload": f"rpCholesky-QR row-sharded FP64 m={m} n={n} s={s} kappa={args.kappa:g} "
                               f"over {ws} process(es)", "m": m, "n": n, "s": s, "kappa": args.kappa,
                   "parallelism": f"rows{ws}", "l2": f"inputs larger than L2 (A = {8 * m * n / 1e9:.2f} GB)"},
        "effective_tflops": alg_flops(m, n, s) * value / 1e12, "status": st,
        "clocks": clk.summary(), "gpu_launches": None, "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(out), flush=True)
    return 0


def batch_inputs(args, torch, dev, rank):
    import inputs
    man = inputs.batch_manifest(args.count, args.seed + 1000 * rank)
    As = [inputs.usv_torch(e["m"], e["n"], e["kappa"], e["seed"], dev) for e in man]
    return man, As, [e["s"] for e in man], [e["seed"] for e in man]


def batch_measure(kind, args, rq, torch, local, dev, dist, man, As, ss, seeds, K, W, clocks=False):
    """The whole batch per step, K timed replays of one captured CUDA graph after W: kind "persistent"
    (rpcholqr_factor_batched, one persistent FP64 kernel launch), "split" or "fp64" (the slot plans of a
    batch object, concurrent streams, slot count autotuned).  Returns (ms per step, Qs, Rs, info, extra)."""
    stream = torch.cuda.current_stream(dev)
    max_m = max(e["m"] for e in man)
    max_n = max(e["n"] for e in man)
    max_s = max(ss)
    extra = {}
    if kind == "persistent":
        owner = rq.rpcholqr_plan_create(local, max_m, max_n, max_s, mode=rq.FP64)
        rq.rpcholqr_plan_set_option(owner, rq.OPT_BATCH_CAPACITY, len(As))
        Qs, Rs, info, arrays = rq.rpcholqr_factor_batched(owner, As, ss, seeds, stream=stream)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                rq.rpcholqr_factor_batched(owner, As, ss, seeds, Qs=Qs, Rs=Rs, info=info, stream=cs, arrays=arrays)
        stream.wait_stream(cs)
        replay = g.replay
        extra["launches_per_step"] = 2
    else:
        owner = rq.rpcholqr_batch_create(local, max_m, max_n, max_s, slots=args.slots,
                                         mode=rq.SPLIT64 if kind == "split" else rq.FP64)
        slots, tune_ms = rq.rpcholqr_batch_autotune(owner, As, ss, seeds, reps=1, stream=stream)
        Qs, Rs, info = rq.rpcholqr_batch_capture(owner, As, ss, seeds, stream=stream)
        replay = lambda: rq.rpcholqr_batch_replay(owner, stream=stream)
        extra.update({"slots": slots, "autotune_ms": tune_ms})
    for _ in range(W):
        replay()
    torch.cuda.synchronize(dev)
    st = info.cpu().view(-1, 2)[:, 0]
    if int((st != 0).sum()) != 0:
        raise RuntimeError(f"batch statuses {st.tolist()}")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with (ClockSampler(local) if clocks else _NoClock()) as clk:
        barrier(dist)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(K):
            replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    extra["clocks"] = clk.summary()
    extra["owner"] = owner
    return max_over_ranks(e0.elapsed_time(e1), dist, dev) / K, Qs, Rs, info, extra


def batch_gate(man, As, Qs, Rs, count=8):
    """Largest orthogonality error over the `count` members with the largest kappa."""
    return max(gpu_metrics(As[i], Qs[i], Rs[i])[0] for i in sorted(range(len(man)), key=lambda j: -man[j]["kappa"])[:count])


def run_config4(args, rq, torch, local, dev, dist, ws):
    """The 512-matrix heterogeneous batch: the persistent FP64 kernel and the SPLIT64 slot graph."""
    man, As, ss, seeds = batch_inputs(args, torch, dev, 0)
    out = {"workload": f"rpCholesky-QR batch of {len(man)} (m log-uniform 4096..2^20, n in {{8,16,32,64,128}}, "
                       f"s=3n, kappa log-uniform 1..1e14), one CUDA-graph replay per step", "count": len(man),
           "l2": "inputs larger than L2 (%.1f GB in total), no flush" % (8 * sum(e["m"] * e["n"] for e in man) / 1e9)}
    flops = sum(alg_flops(e["m"], e["n"], e["s"]) for e in man)
    for kind in ("persistent", "split"):
        ms, Qs, Rs, info, extra = batch_measure(kind, args, rq, torch, local, dev, dist, man, As, ss, seeds,
                                                max(3, args.steps // 4), 2)
        owner = extra.pop("owner")
        orth = None if args.no_metrics else batch_gate(man, As, Qs, Rs)
        owner.close()
        out[kind] = {"mode": "fp64" if kind == "persistent" else "split",
                     "launch": "one persistent kernel (rpcholqr_factor_batched)" if kind == "persistent" else
                               "16 slot plans on concurrent streams (rpcholqr_batch_*)",
                     "value": ws * len(man) / (ms / 1e3), "unit": "matrices/s", "ms_per_step": ms,
                     "effective_tflops": flops / (ms / 1e3) / 1e12, "orth_max_sampled": orth,
                     **{k: v for k, v in extra.items() if k != "clocks"}}
        del Qs, Rs
        torch.cuda.empty_cache()
    del As
    torch.cuda.empty_cache()
    return out


def run_batch(args, ws, rank, local):
    """The heterogeneous batch: one step = the whole batch, replayed from one captured CUDA graph; the
    split mode runs the slot plans, the FP64 mode the persistent kernel."""
    import torch

    import paper_2406_11751_gb300 as rq

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(ws, "nccl")
    rq.build()
    preload_torch_linalg()
    K, W = args.steps, args.warmup
    man, As, ss, seeds = batch_inputs(args, torch, dev, rank)
    fp64_peak = rq.rpcholqr_probe_fp64_mma(local, 4096)
    kind = "split" if args.mode == "split" else "persistent"
    ms, Qs, Rs, info, extra = batch_measure(kind, args, rq, torch, local, dev, dist, man, As, ss, seeds, K, W,
                                            clocks=True)
    owner = extra.pop("owner")
    clk = extra.pop("clocks")
    orth = batch_gate(man, As, Qs, Rs)
    owner.close()
    if rank != 0:
        return 0
    count = len(man)
    value = ws * count / (ms / 1e3)
    flops = sum(alg_flops(e["m"], e["n"], e["s"]) for e in man)
    if args.mode == "fp64":
        fp64_work = flops
    else:
        # split mode: the FP64 row solves of the 32-column diagonal blocks, m * sum_J b_J^2 flop per matrix
        fp64_work = float(sum(e["m"] * sum(min(32, e["n"] - c) ** 2 for c in range(0, e["n"], 32)) for e in man))
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        # oracle on four batch members, each on a bounded row sample; per-matrix time scaled by rows
        import inputs
        import oracle
        oracle.build()
        sample = sorted(man, key=lambda e: e["m"])[::len(man) // 4][:4]
        per_row = []
        for e in sample:
            rows = min(e["m"], 1 << 15)
            Ah = inputs.usv(rows, e["n"], e["kappa"], e["seed"])
            t0 = time.perf_counter()
            oracle.rpcholqr(Ah, min(e["s"], rows), e["seed"])
            per_row.append(((time.perf_counter() - t0) / (rows * e["n"] * e["n"])))
        c_row = sum(per_row) / len(per_row)
        tot = sum(c_row * e["m"] * e["n"] * e["n"] for e in man)
        cpu = {"value": count / tot, "unit": "matrices/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "oracle on 4 batch members (rows capped at 32768), time per m n^2 averaged and "
                         "summed over the 512 shapes"}
    out = {
        "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "split": "f64+bf16", "fp32": "f32+f64"}[args.mode],
        "data": "synthetic (A = U diag(sigma) V^T per manifest entry, Haar U/V from torch)",
        "config": {"workload": f"rpCholesky-QR batch of {count} (m log-uniform 4096..2^20, n in "
                               f"{{8,16,32,64,128}}, s=3n, kappa log-uniform 1..1e14), {args.mode.upper()}, "
                               f"one CUDA-graph replay per step ("
                               + ("one persistent kernel" if kind == "persistent" else "slot plans") + ")",
                   "count": count, "mode": args.mode, **{k: v for k, v in extra.items()},
                   "l2": "inputs larger than L2 (%.1f GB in total), no flush" %
                         (8 * sum(e["m"] * e["n"] for e in man) / 1e9)},
        "effective_tflops": flops / (ms / 1e3) / 1e12,
        "orth_max_sampled": orth, "gate_orth_le_1e-13": bool(orth <= 1e-13),
        "roofline": {"kernel": "whole batch: " + ("all FP64 work (row passes dominate)" if args.mode == "fp64" else
                                                  "the FP64-pipe work (32-column diagonal-block row solves; "
                                                  "the products run on the tensor cores)"),
                     "bound": "alu",
                     "achieved": fp64_work / (ms / 1e3) / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                     "frac": fp64_work / (ms / 1e3) / fp64_peak, "traffic": None,
                     "note": "algorithmic flops of that work over the whole replay time (every other kernel "
                             "included in the time)"},
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": extra.get("launches_per_step"),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "batch":
        return run_batch(args, ws, rank, local)
    if args.sharded:
        return run_sharded(args, ws, rank, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
