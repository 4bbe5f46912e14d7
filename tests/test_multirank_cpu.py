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


# ---- query sharding (paper_1511_02186_gb300.sharding) ----------------------------------------

def test_query_ranges_cover_every_query_once():
    from paper_1511_02186_gb300.sharding import query_ranges
    for m in (0, 1, 2, 7, 1000, 1 << 20, 1048577):
        for world in (1, 2, 3, 4, 7, 8):
            rs = query_ranges(m, world)
            assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [e - b for b, e in rs]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        query_ranges(5, 0)


def _shard_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    from paper_1511_02186_gb300 import sharding, workloads
    bench.dist_setup(world)
    wl = workloads.small_case(41, 3000, 1001, k=7, pattern="clustered")

    def compute(a, b):  # the per-rank compute of this test: the oracle on the rank's slice
        r = oracle.interpolate(wl.x, wl.y, wl.z, wl.area, a, b, wl.k, threads=1)
        return {"z": r["z"], "alpha": r["alpha"], "knn": r["knn"]}

    b, e, own = sharding.shard_interpolate(compute, wl.qx, wl.qy, rank, world, gather=False)
    b0, e0, full = sharding.shard_interpolate(compute, wl.qx, wl.qy, rank, world, gather=True)
    q.put((rank, b, e, b0, e0, {k: v.tolist() for k, v in full.items()}))
    dist.destroy_process_group()


def test_sharded_results_equal_the_single_rank_result():
    """Two gloo ranks each interpolate their contiguous range of 1,001 queries (the oracle as
    the per-rank compute); the gathered arrays equal the one-rank result element for element,
    in the caller's order."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_1511_02186_gb300 import workloads
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = workloads.small_case(41, 3000, 1001, k=7, pattern="clustered")
    ref = oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx, wl.qy, wl.k, threads=1)
    assert [(g[1], g[2]) for g in got] == [(0, 501), (501, 1001)]
    for rank, b, e, b0, e0, full in got:
        assert (b0, e0) == (0, wl.m)
        assert np.array_equal(np.asarray(full["z"]), ref["z"])
        assert np.array_equal(np.asarray(full["alpha"]), ref["alpha"])
        assert np.array_equal(np.asarray(full["knn"]), ref["knn"])
