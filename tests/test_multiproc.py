"""The multi-rank host logic of bench.py on CPU with the gloo backend, world size 2.

Every rank of a multi-GPU run is an independent replica (no data-path collective); the only
exchange is the timing: the job's rate is all ranks' units over the slowest rank's time.  The
reference arm (the FP64 oracle on the host) runs on rank 0 alone, the other ranks exit 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    # rank 1 is the slow one: 3 s for its 10 steps against rank 0's 1 s
    rate, slowest = bench.job_rate(10, 1.0 + 2.0 * rank, 2, "cpu")
    worst = bench.max_over_ranks(5.0 - rank, 2, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rate": rate, "slowest": slowest, "worst": worst}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_all_units_over_the_slowest_rank(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["slowest"] == 3.0
        assert got["rate"] == pytest.approx(20 / 3.0)
        assert got["worst"] == 5.0


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(7, 2.0, 1, "cpu") == (3.5, 2.0)


def test_reference_arm_runs_on_rank_zero_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-seconds", "1",
           "--workload", "par2d_128_ffn64"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
