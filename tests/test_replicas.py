"""The multi-GPU path of bench.py on the CPU: replicas over gloo (world size 2).

Frames are independent, so N GPUs run N replicas; the only collective is the max of
the per-rank step times.  These tests run the rank logic and a full torchrun launch of
the CPU reference arm without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        out[rank] = (bench.max_over_ranks(dist, ms), bench.frame_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_distinct_frames_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0     # every rank reports the slowest time
    assert res[0][1] != res[1][1]             # each replica decodes its own frames


def test_reference_arm_under_torchrun_world_2():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--ref-frames", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                     # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_bench_code_choices_resolve():
    # every --code name loads a committed code, and the workload line names its sizes
    import argparse

    sys.path.insert(0, ROOT)
    import bench
    from paper_2305_05286_gb300 import inputs as I

    for name in bench.CODES:
        qc = bench.bench_code(I, name)
        args = argparse.Namespace(code=name, frames=1000, ebn0=2.5, alg="cbp_sp", gpus=1)
        cfg = bench.workload_config(args, qc)
        assert f"N={qc.N}" in cfg["workload"] and bench.CODES[name][1] in cfg["workload"]
        assert "within L2" in cfg["l2"] or "larger than L2" in cfg["l2"]
    qc = bench.bench_code(I, "26112")
    big = argparse.Namespace(code="26112", frames=65536, ebn0=2.5, alg="cbp_sp", gpus=1)
    assert "6.85 GB" in bench.workload_config(big, qc)["l2"]
