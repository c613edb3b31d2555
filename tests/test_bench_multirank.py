"""bench.py's multi-process host logic on CPU ranks (gloo, world size 2): the max-over-ranks timing,
the barrier, and the reference arm's rank-0-only output."""
import io
import os
import socket
import sys
import tempfile
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_env()
    dist = bench.init_dist(ws, "gloo")
    try:
        t = bench.max_over_ranks(10.0 + 5 * r, dist)       # rank 1 is the slowest
        bench.barrier(dist)
        # the reference arm: rank 0 prints one line, the others return 0 without work
        sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "0",
                    "--m", "300", "--n", "4", "--cpu-sample-rows", "300"]
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.main()
        with open(os.path.join(outdir, f"r{r}.txt"), "w") as f:
            f.write(f"{t}\n{rc}\n{buf.getvalue()}")
    finally:
        dist.destroy_process_group()


def test_bench_rank_logic_world2():
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        outs = [open(os.path.join(d, f"r{r}.txt")).read().split("\n", 2) for r in range(2)]
    assert [float(o[0]) for o in outs] == [15.0, 15.0]
    assert [int(o[1]) for o in outs] == [0, 0]
    assert '"impl": "reference"' in outs[0][2] and outs[0][2].count("\n") == 1
    assert outs[1][2] == ""


def test_traffic_from_profiles_scales_and_checks_source(tmp_path, monkeypatch):
    # a class's recorded DRAM bytes (one call's total at the captured rows) are used only for an unchanged
    # kernel source, scaled from the captured row count to the run's and split over the call's launches
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(
        "# class=split_gemm n=512 src_sha=" + sha + " dram_bytes_per_call=1 measured_m=1 (a comment)\n"
        f"class=split_gemm n=512 src_sha={sha} dram_bytes_per_call=1000 measured_m=1024\n"
        f"class=split_gemm n=128 src_sha={sha} dram_bytes_per_call=64 measured_m=1024\n"
        "class=rowpass n=512 src_sha=0000000000000000 dram_bytes_per_call=5 measured_m=1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("split_gemm", 512, str(src), 1024, 1) == 1000.0
    assert bench.traffic_from_profiles("split_gemm", 512, str(src), 4096, 8) == 500.0
    assert bench.traffic_from_profiles("split_gemm", 128, str(src), 2048, 2) == 64.0
    assert bench.traffic_from_profiles("rowpass", 512, str(src), 1, 1) is None        # source changed
    assert bench.traffic_from_profiles("split_gram", 512, str(src), 1, 1) is None     # never captured
