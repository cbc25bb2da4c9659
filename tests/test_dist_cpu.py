"""The multi-process (replica) path on CPU: gloo, world size 2.

Every rank runs its own lattice (seed + rank) with no data-path collective;
the only collectives are the benchmark's barrier and the max over ranks of
the timed region. These tests run those helpers and the reference arm of
bench.py under two local processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench._barrier(world)
    v = bench._max_over_ranks(world, 1.5 + rank)
    bench._barrier(world)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"max": v}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / ("rank%d.json" % r)))["max"] for r in range(2)]
    assert got == [2.5, 2.5]


def test_reference_arm_under_torchrun(tmp_path):
    """bench.py --impl reference at N = 2: rank 0 prints one JSON line, the
    other rank exits 0 without output."""
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node",
           "2", "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
