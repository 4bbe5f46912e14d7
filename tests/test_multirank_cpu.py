"""Multi-process checks of bench.py's N > 1 plumbing on CPU with the gloo backend (world size 2):
process-group set-up from the torchrun environment, the barrier, the max-over-ranks timing
reduction, and the reference arm printing one line from rank 0 only."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup(world)
    assert dist.get_backend() == "gloo"
    # Each rank "timed" a different duration; every rank must see the slowest.
    t = bench.max_over_ranks(0.25 + rank, w, torch.device("cpu"))
    bench.barrier(w)
    q.put((r, w, local, t))
    dist.destroy_process_group()


def test_dist_setup_barrier_and_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(g[0] for g in got) == [0, 1]
    assert all(g[1] == world and g[2] == g[0] for g in got)
    assert all(g[3] == pytest.approx(1.25) for g in got)


def test_single_process_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(1) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    bench.barrier(1)


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    obj = json.loads(lines[0])
    assert obj["impl"] == "reference" and obj["n_gpus"] == 2
    assert obj["value"] > 0 and obj["cpu_baseline"]["kind"] == "oracle"
    assert obj["e2e"]["h2d_bytes_per_step"] == 0
