"""The multi-GPU form of the benchmark: independent replicas, one per rank.

The product shards into independent problems, so ranks exchange nothing on the data
path; the only collective is the timing reduction (the job's time is its slowest
rank's).  These run on the CPU: the reduction over two gloo ranks, the per-rank
inputs, and the reference arm launched by torchrun (rank 0 alone reports).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.reduce_max(1.5 + 2.0 * rank, ws, torch.device("cpu"))
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(repr(got))
    finally:
        tdist.destroy_process_group()


def test_slowest_rank_time_reaches_every_rank(tmp_path):
    import torch.multiprocessing as tmp
    ws, port = 2, _free_port()
    tmp.spawn(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    got = [float((tmp_path / f"r{r}.txt").read_text()) for r in range(ws)]
    assert got == [3.5, 3.5]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(7.25, 1, None) == 7.25


def test_ranks_draw_their_own_seeded_inputs():
    sys.path.insert(0, ROOT)
    import bench
    a0, b0, _ = bench.make_inputs("c1_256_p256", 0)
    a0b, b0b, _ = bench.make_inputs("c1_256_p256", 0)
    a1, b1, _ = bench.make_inputs("c1_256_p256", 1)
    assert np.array_equal(a0.limb, a0b.limb) and np.array_equal(b0.limb, b0b.limb)   # deterministic per rank
    assert not np.array_equal(a0.limb, a1.limb) and not np.array_equal(b0.limb, b1.limb)   # own matrices


def test_reference_arm_under_torchrun_reports_once(tmp_path):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "c2_1024_p512", "--cpu-seconds", "0.5"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_of_the_batched_workload():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c3_batch64",
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"].startswith("c3_batch64")
