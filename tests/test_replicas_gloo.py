"""Multi-process paths of the benchmark on the CPU (gloo, world size 2).

The solves do not shard: N GPUs run N independent replicas with no
collective on the data path.  What crosses ranks is the timing (the slowest
rank's time, combined into a whole-job rate) and, for the reference arm under
torchrun, the rule that rank 0 alone runs and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms_local = [12.5, 20.0][rank]                  # rank 1 is the slower replica
    ms = bench.max_over_ranks(dist, ms_local, "cpu")
    q.put((rank, ms, bench.replica_value(world, 100, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_whole_job_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, val in got:
        assert ms == 20.0                          # max over ranks, seen by both
        assert val == pytest.approx(2 * 100 / 0.020)
    import bench
    assert bench.max_over_ranks(None, 7.0, "cpu") == 7.0


def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference launched with torchrun on two ranks: rank 0
    runs the oracle and prints one JSON line, rank 1 exits 0 without work."""
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--p", "1"]
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
