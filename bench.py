"""AIDW benchmark: pair-evaluations per second of the FP32-compensated path on GB300.

Workload (one step): AIDW of 1,048,576 query points against 1,048,576 data points, uniform in
[0,1000]^2 (A = 1e6), z = sin(x/100) + cos(y/150) + 0.05 N(0,1), k = 10, levels (1,2,3,4,5),
R_min = 0, R_max = 2 -- the paper's largest size class (Sec. 4: as many queries as data points,
uniform in a square), seeded synthetic data. A pair-evaluation is one (query, data point) pair
carried through both phases (kNN scan and weighted sum); a step is n * m of them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--scaling S]
Prints one JSON line (rank 0). Under torchrun the queries are sharded over the ranks, each rank
holding a replica of the dataset on its own GPU (queries are independent; no collective on the
data path): with --scaling weak (the default) every rank interpolates its own 1,048,576
queries, with --scaling strong the workload's queries are split into contiguous ranges. The
value is all ranks' pair-evaluations over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AIDW pair-evals/s (FP32-compensated path)"
UNIT = "pair-evals/s"
N_DATA = 1 << 20
M_QUERY = 1 << 20
L2_FLUSH_BYTES = 256 << 20
# Algorithmic work per pair-evaluation. Phase 2 (Eq. 1 over all n points) needs, per pair,
# 2 sub, 1 mul, 1 fma (squared distance), 1 fma (power scale), 1 add, 1 fma (the two sums) and
# one MUFU lg2 plus one MUFU ex2. Phase 1 is exact but pruned (nearest-first tiles with
# bounding-box bounds), so it has no per-pair minimum; a step's n * m pair-evaluations are bound
# by phase 2.
FP32_OPS_P2, MUFU_OPS_P2 = 7, 2
FP64_OPS_P2 = 6  # FP64 instructions per pair in the FP64 phase-2 kernel
FP64X_OPS_P2 = 4  # FP64 instructions per pair in the AIDW_F64X phase-2 kernel (the distance)
FP64_PIPE_PER_CLK_SM = 2.0  # GB300 FP64 pipe: 1.25 TFLOP/s nominal = 2 DFMA per clk per SM
LANES_PER_SM = 128  # FP32 lanes and issue slots (4 schedulers x 32) per SM per clock


def source_digest(path: str) -> str:
    """SHA-1 of a C++ source with comments and whitespace removed: edits to comments alone do
    not change it, any change to the code does."""
    import hashlib
    import re
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha1(" ".join(text.split()).encode()).hexdigest()


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` (the template instance the timed step launches) from
    the committed ncu capture, or None when the capture is of another instance or the code of
    the kernel's sources changed since (the counters would no longer describe it)."""
    path = os.path.join(ROOT, "profiles", "weights_kernel_traffic_uniform_1Mx1M.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec["kernel"] != kernel:
            return None
        for rel, digest in rec["source_digest"].items():
            if source_digest(os.path.join(ROOT, rel)) != digest:
                return None
        return rec["dram_read_bytes"] + rec["dram_write_bytes"]
    except (OSError, KeyError, ValueError):
        return None


def workload_config(wl):
    name = "uniform_paper_1M_x_1M" if wl.n == N_DATA and wl.m == M_QUERY else \
        f"uniform_paper_{wl.n}_x_{wl.m}"
    return {"workload": name, "n_data": wl.n, "m_query": wl.m, "k": wl.k,
            "levels": list(wl.levels), "r_min": wl.r_min, "r_max": wl.r_max, "area": wl.area,
            "domain": "[0,1000]^2", "seed": 0,
            "l2": "flushed between timed steps by a 256 MiB write (outside the timed events)"}


def rank_workload(wl, rank: int, world: int, scaling: str):
    """This rank's queries against the replicated dataset. Strong scaling: its contiguous range
    of the workload's queries (query_ranges). Weak scaling: a full query set of its own (rank 0
    the workload's, rank r > 0 fresh seeded uniform points in the same square), so that every
    rank does the same amount of work as N grows."""
    import dataclasses
    from paper_1511_02186_gb300.sharding import query_ranges
    if world == 1:
        return wl
    if scaling == "strong":
        b, e = query_ranges(wl.m, world)[rank]
        return wl.query_subset(np.arange(b, e))
    if rank == 0:
        return wl
    rng = np.random.default_rng(1000 + rank)
    side = float(np.sqrt(wl.area))
    return dataclasses.replace(wl, qx=rng.uniform(0.0, side, wl.m), qy=rng.uniform(0.0, side, wl.m))


# ---- clocks ------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [s.strip() for s in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- distributed plumbing -------------------------------------------------------------------

def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- CPU baseline (the FP64 oracle, as it stands) --------------------------------------------

def oracle_rate(wl, target_s: float, threads: int):
    """Times the oracle on a seeded query sample sized for about target_s seconds of CPU work;
    returns (pair-evals/s, sample description, threads)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(123)
    q = 64
    idx = rng.choice(wl.m, q, replace=False)
    t0 = time.perf_counter()
    oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx[idx], wl.qy[idx], wl.k, wl.levels,
                       threads=threads)
    dt = time.perf_counter() - t0
    q2 = int(min(wl.m, max(q, q * target_s / max(dt, 1e-3))))
    q2 = max(threads, (q2 // threads) * threads)
    idx = rng.choice(wl.m, q2, replace=False)
    t0 = time.perf_counter()
    oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx[idx], wl.qy[idx], wl.k, wl.levels,
                       threads=threads)
    dt = time.perf_counter() - t0
    return (q2 * wl.n) / dt, f"{q2} seeded queries x all {wl.n} data points, {dt:.1f} s", threads


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    from paper_1511_02186_gb300 import workloads
    wl = workloads.uniform_paper(0)
    threads = os.cpu_count() or 1
    vals = []
    for _ in range(args.warmup):
        oracle_rate_small(wl, threads)
    for _ in range(args.steps):
        vals.append(oracle_rate_small(wl, threads))
    v = statistics.median([x[0] for x in vals])
    sample = vals[0][1]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median([x[2] for x in vals]) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def oracle_rate_small(wl, threads):
    import oracle
    rng = np.random.default_rng(len(wl.qx))
    q = 8 * threads
    idx = rng.choice(wl.m, q, replace=False)
    t0 = time.perf_counter()
    oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx[idx], wl.qy[idx], wl.k, wl.levels,
                       threads=threads)
    dt = time.perf_counter() - t0
    return q * wl.n / dt, f"{q} seeded queries x all {wl.n} data points per step", dt


# ---- batched and served configurations -------------------------------------------------------

def bench_batched(ctx, steps: int, warmup: int, dev, stream, tune: bool = True, peak=None):
    """256 independent datasets (n log-uniform in [1,024, 262,144], m log-uniform in
    [1,024, 65,536], side log-uniform in [10, 1000], uniform or clustered, k in {6, 10, 15}) in
    one persistent launch replayed from a CUDA graph: timed with the built-in kernel shape,
    then (with `tune`) autotuned on the batch itself and timed again with the winning shape."""
    import torch
    from paper_1511_02186_gb300 import aidw, workloads
    wls = workloads.batched(0)
    items = []
    for wl in wls:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device=dev)
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device=dev)
        out = torch.empty(wl.m, dtype=torch.float32, device=dev)
        items.append((ds, qx, qy, aidw.default_params(k=wl.k), out, None))
    pairs = float(sum(wl.n * wl.m for wl in wls))
    pb = ctx.batch_create(items)

    def timed():
        for _ in range(max(1, warmup)):
            pb.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for a, b in evs:
            a.record(stream)
            pb.launch(stream.cuda_stream)
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in evs)

    ms_default = timed()
    t0 = time.perf_counter()
    if tune:
        cfg, tune_ms = pb.autotune(reps=2)
        ms = timed()
    else:
        cfg, ms = pb.config(), ms_default
    tune_s = time.perf_counter() - t0
    pb.destroy()
    for it in items:
        it[0].destroy()
    return {"workload": "batched_256_datasets", "datasets": len(wls),
            "pair_evals_per_launch": pairs, "launches": steps,
            "ms_per_launch": ms,
            "value": pairs / (ms / 1e3), "unit": UNIT,
            "queries": int(sum(wl.m for wl in wls)),
            "tuned_config": cfg.as_dict(), "autotune_s": tune_s,
            "default_config_ms_per_launch": ms_default,
            "default_config_value": pairs / (ms_default / 1e3),
            "frac_of_phase2_bound": None if peak is None else pairs / (ms / 1e3) / peak,
            "phase2_bound": peak,
            "launch": "one persistent work-queue kernel per batch, replayed from a CUDA graph; "
                      "kernel shape chosen by the autotuner on this batch"}


def bench_standard_idw(ctx, ds, wl, dev, stream, peak):
    """Standard IDW (Eq. 1 with one constant power, the paper's comparison method) on the 1M
    dataset for 262,144 seeded queries, FP32 path: one warm-up and three timed calls of
    aidw_idw (a one-neighbour phase 1 for the normalising distance and the coincidence test,
    then phase 2 over all points), reported against the phase-2 bound."""
    import torch
    from paper_1511_02186_gb300 import aidw
    q = 262144
    idx = torch.as_tensor(np.random.default_rng(11).choice(wl.m, q, replace=False))
    qx = torch.as_tensor(wl.qx, dtype=torch.float32, device=dev)[idx.to(dev)].contiguous()
    qy = torch.as_tensor(wl.qy, dtype=torch.float32, device=dev)[idx.to(dev)].contiguous()
    out = torch.empty(q, dtype=torch.float32, device=dev)
    ctx.idw(ds, qx, qy, 2.0, aidw.F32C, out=out, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        ctx.idw(ds, qx, qy, 2.0, aidw.F32C, out=out, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    value = q * wl.n / (ms / 1e3)
    return {"workload": f"uniform_{wl.n}_x_{q}", "power": 2.0, "precision": "f32",
            "ms": ms, "value": value, "unit": UNIT, "frac_of_phase2_bound": value / peak}


SERVED_BUCKETS = ((256, 4096), (4096, 65536), (65536, 262145))


def latency_summary(lat_ms, ms_):
    """p50 / p99 / max of request latencies, overall and per query-count bucket."""
    lat_ms, ms_ = np.asarray(lat_ms), np.asarray(ms_)
    out = {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
           "max_ms": float(lat_ms.max())}
    by = {}
    for lo, hi in SERVED_BUCKETS:
        sel = (ms_ >= lo) & (ms_ < hi)
        if sel.any():
            by[f"{lo}-{hi - 1}_queries"] = {
                "requests": int(sel.sum()), "p50_ms": float(np.percentile(lat_ms[sel], 50)),
                "p99_ms": float(np.percentile(lat_ms[sel], 99))}
    out["by_request_size"] = by
    return out


def bench_served(ctx, capacity_pairs_s: float, requests_per_level: int, nominal_window_s: float,
                 nominal_queue: int):
    """64 resident datasets (n log-uniform in [16K, 1M]); Poisson arrivals of requests with
    256..262,144 query points (log-uniform, host arrays) uniform in the dataset's square.
    Runs at 0.25, 0.5 and 0.8 of the measured single-launch capacity (about
    `requests_per_level` requests each; a refused submit is retried after 1 ms) and at the
    nominal 2,000 req/s over `nominal_window_s` seconds, an offered load several times the
    capacity, against a serving queue of `nominal_queue` requests: a submit refused with
    AIDW_ERR_AGAIN is shed (counted, not retried), which is the backpressure a client sees.
    Latencies are reported overall and per request-size bucket. Then serves a prefix of a
    request stream one request per launch (FP64 and FP32, no batching) for comparison."""
    from paper_1511_02186_gb300 import aidw, workloads
    dsw = workloads.served_datasets(0)
    handles = [ctx.create_dataset(w.x, w.y, w.z, w.area) for w in dsw]
    pool = workloads.served_query_pool(dsw)
    p = aidw.default_params(k=10)
    probe = workloads.served_arrivals(dsw, seed=11, rate=2000.0, duration_s=1.0)
    mean_pairs = statistics.mean(dsw[d].n * m for _, d, m in probe)
    results = {"mean_pair_evals_per_request": mean_pairs,
               "queries": "slices of a per-dataset pool of 262,144 seeded uniform points"}
    runs = []
    for i, f in enumerate((0.25, 0.5, 0.8)):
        rate = max(1.0, f * capacity_pairs_s / mean_pairs)
        runs.append((f"load_{f:.2f}_of_capacity", rate, requests_per_level / rate, 12 + i, 0))
    runs.append(("nominal_2000_per_s", 2000.0, nominal_window_s, 20, nominal_queue))
    rng = np.random.default_rng(21)
    for label, rate, window, seed, queue in runs:
        arrivals = workloads.served_arrivals(dsw, seed=seed, rate=rate, duration_s=window)
        if queue:
            ctx.serving_set_queue_limit(queue)
        ids = []
        again = shed = 0
        t0 = time.perf_counter()
        for t, d, m in arrivals:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            off = int(rng.integers(0, len(pool[d][0]) - m + 1))
            qx, qy = pool[d][0][off:off + m], pool[d][1][off:off + m]
            out = np.empty(m, dtype=np.float32)
            while True:
                rc, rid = ctx.submit(handles[d], qx, qy, p, out)
                if rc != aidw.ERR_AGAIN:
                    break
                again += 1
                if queue:
                    break  # shed
                time.sleep(0.001)
            if rc == aidw.ERR_AGAIN:
                shed += 1
                continue
            ids.append((rid, dsw[d].n * m, m))
        t_submitted = time.perf_counter() - t0
        for rid, _, _ in ids:
            ctx.wait(rid, -1)
        wall = time.perf_counter() - t0
        lat = np.array([ctx.latency_us(rid) for rid, _, _ in ids]) / 1e3
        for rid, _, _ in ids:
            ctx.release(rid)
        if queue:
            ctx.serving_set_queue_limit(4096)
        pairs = float(sum(x for _, x, _ in ids))
        results[label] = {"rate_req_per_s": rate, "window_s": window, "offered_requests":
                          len(arrivals), "requests": len(ids),
                          **latency_summary(lat, [m for _, _, m in ids]),
                          "throughput": pairs / wall, "unit": UNIT,
                          "offered": rate * mean_pairs, "refused_again": again,
                          "shed": shed, "queue_limit": queue or 4096,
                          "submit_phase_s": t_submitted, "wall_s": wall}
    results["sustained"] = results["load_0.50_of_capacity"]
    st = ctx.serving_stats()
    results["launches"] = int(st.launches)
    results["max_concurrent_launches"] = int(st.max_concurrent_launches)
    results["mean_requests_per_launch"] = st.batched_requests / max(1, st.launches)
    results["rejected_again_total"] = int(st.rejected_again)
    results["workload"] = "served_64_datasets_poisson"

    # One set of requests served three ways with nothing else running: one synchronous call per
    # request in FP64 and in FP32 (unbatched), and all of them submitted at once (batched FP32).
    # The set: requests of a seeded stream in arrival order, skipping any that would take the
    # total above 4e10 pair-evaluations (a few seconds of FP64 work), at most 32.
    subset, acc = [], 0.0
    for _, d, qx, qy in workloads.served_requests(dsw, seed=13, rate=1000.0, duration_s=2.0):
        pe = float(dsw[d].n * len(qx))
        if acc + pe > 4e10:
            continue
        subset.append((d, qx, qy))
        acc += pe
        if len(subset) == 32:
            break
    cmp = {"requests": len(subset), "pair_evals": acc,
           "selection": "seeded request stream in arrival order, skipping requests that would "
                        "take the total above 4e10 pair-evaluations, at most 32"}
    for label, prec in (("unbatched_fp64", aidw.F64), ("unbatched_fp32", aidw.F32C)):
        pp = aidw.default_params(k=10, precision=prec)
        dt = np.float64 if prec == aidw.F64 else np.float32
        reqs = [(d, qx.astype(dt), qy.astype(dt), np.empty(len(qx), dtype=dt))
                for d, qx, qy in subset]
        svc = []
        t0 = time.perf_counter()
        for d, qx, qy, out in reqs:
            t1 = time.perf_counter()
            ctx.interpolate(handles[d], qx, qy, pp, out=out)
            svc.append(time.perf_counter() - t1)
        wall = time.perf_counter() - t0
        svc_ms = np.array(svc) * 1e3
        cmp[label] = {"throughput": acc / wall, "unit": UNIT, "wall_s": wall,
                      "p50_service_ms": float(np.percentile(svc_ms, 50)),
                      "p99_service_ms": float(np.percentile(svc_ms, 99)),
                      "launch": "one aidw_interpolate per request, host arrays, back to back"}
    reqs = [(d, qx.astype(np.float32), qy.astype(np.float32), np.empty(len(qx), np.float32))
            for d, qx, qy in subset]
    t0 = time.perf_counter()
    ids = [ctx.submit(handles[d], qx, qy, p, out)[1] for d, qx, qy, out in reqs]
    for rid in ids:
        ctx.wait(rid, -1)
    wall = time.perf_counter() - t0
    lat = np.array([ctx.latency_us(rid) for rid in ids]) / 1e3
    for rid in ids:
        ctx.release(rid)
    cmp["batched_fp32_burst"] = {"throughput": acc / wall, "unit": UNIT, "wall_s": wall,
                                 "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)),
                                 "launch": "all requests submitted at once to the serving "
                                           "runtime (continuous batching)"}
    results["same_requests_batched_vs_unbatched"] = cmp
    for h in handles:
        h.destroy()
    return results


def bench_paper_designs(ctx, dev, stream, n: int = 262144, n64: int = 32768):
    """The paper's kernel designs (naive / tiled x SoA / AoaS, Sec. 3.1) against the optimized
    path on uniform workloads in [0,1000]^2 with k = 10 and m = 262,144 queries (enough
    one-thread-per-query blocks to fill every SM): FP32 with n = 262,144 data points, FP64 with
    n64 = 32,768. Each variant runs once on 1,024 queries (warm-up), then once timed."""
    import torch
    from paper_1511_02186_gb300 import aidw, workloads
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    names = {(aidw.VERSION_NAIVE, aidw.LAYOUT_SOA): "naive_soa",
             (aidw.VERSION_NAIVE, aidw.LAYOUT_AOAS): "naive_aoas",
             (aidw.VERSION_TILED, aidw.LAYOUT_SOA): "tiled_soa",
             (aidw.VERSION_TILED, aidw.LAYOUT_AOAS): "tiled_aoas"}
    for prec, label, nd in ((aidw.F32C, "fp32", n), (aidw.F64, "fp64", n64)):
        wl = workloads.uniform_paper(0, n=nd, m=n)
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        dt = torch.float64 if prec == aidw.F64 else torch.float32
        qx = torch.as_tensor(wl.qx, dtype=dt, device=dev)
        qy = torch.as_tensor(wl.qy, dtype=dt, device=dev)
        out = torch.empty(wl.m, dtype=dt, device=dev)
        p = aidw.default_params(k=wl.k, levels=wl.levels, precision=prec)
        pairs = float(wl.m) * wl.n
        row = {"workload": f"uniform_{wl.n}x{wl.m}", "n": wl.n, "m": wl.m, "k": wl.k,
               "pair_evals": pairs}

        def timed(fn):
            fn(qx[:1024], qy[:1024], out[:1024])
            torch.cuda.synchronize()
            e0.record(stream)
            fn(qx, qy, out)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            return {"ms": ms, "value": pairs / (ms / 1e3)}

        for (ver, lay), nm in names.items():
            row[nm] = timed(lambda a, b, o, ver=ver, lay=lay: ctx.interpolate_paper(
                ds, a, b, p, version=ver, layout=lay, out=o, stream=stream.cuda_stream))
        ctx.set_profiling(True)
        row["optimized"] = timed(lambda a, b, o: ctx.interpolate(
            ds, a, b, p, out=o, stream=stream.cuda_stream))
        kt = ctx.kernel_times()
        ctx.set_profiling(False)
        row["optimized"]["kernel_ms"] = {"knn": kt.knn_ms, "select": kt.select_ms,
                                         "weights": kt.weights_ms, "finalize": kt.finalize_ms,
                                         "knn_splits": kt.splits, "w_splits": kt.weight_splits}
        row["tiled_over_naive_soa"] = row["naive_soa"]["ms"] / row["tiled_soa"]["ms"]
        row["soa_over_aoas_naive"] = row["naive_aoas"]["ms"] / row["naive_soa"]["ms"]
        row["soa_over_aoas_tiled"] = row["tiled_aoas"]["ms"] / row["tiled_soa"]["ms"]
        row["optimized_over_tiled_soa"] = row["tiled_soa"]["ms"] / row["optimized"]["ms"]
        res[label] = row
        ds.destroy()
    return res


def bench_precision_stress(ctx, dev, stream):
    """The clustered precision-stress workload: 2,097,152 data points (90 % from 32 Gaussians,
    sigma 5-50, 10 % uniform) in [0,1000]^2, queries on the 1448 x 1448 cell-centre grid,
    z lognormal(0, 1), k = 10. One FP32 launch over all queries (timed), its error against the
    FP64 oracle on 768 queries (256 seeded, plus the 256 smallest and 256 largest alpha), and
    the FP64 GPU path on 2,048 seeded queries."""
    import torch
    import oracle
    from paper_1511_02186_gb300 import aidw, workloads
    wl = workloads.clustered_grid(0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx = torch.as_tensor(wl.qx, dtype=torch.float32, device=dev)
    qy = torch.as_tensor(wl.qy, dtype=torch.float32, device=dev)
    out = torch.empty(wl.m, dtype=torch.float32, device=dev)
    oa = torch.empty(wl.m, dtype=torch.float32, device=dev)
    p = aidw.default_params(k=wl.k, levels=wl.levels)
    ctx.interpolate(ds, qx, qy, p, out=out, out_alpha=oa, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.interpolate(ds, qx, qy, p, out=out, out_alpha=oa, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    z = out.cpu().numpy().astype(np.float64)
    alpha = oa.cpu().numpy()
    order = np.argsort(alpha, kind="stable")
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([rng.choice(wl.m, 256, replace=False), order[:256],
                                    order[-256:]]))
    w32 = wl.as_f32()
    ref = oracle.interpolate(w32.x, w32.y, w32.z, w32.area, w32.qx[idx], w32.qy[idx], w32.k,
                             w32.levels, w32.r_min, w32.r_max)
    den = np.maximum(np.abs(ref["z"]), ref["scale"])
    err = np.abs(z[idx] - ref["z"]) / den
    pure = np.abs(z[idx] - ref["z"]) / np.abs(ref["z"])
    q64 = 2048
    i64 = torch.as_tensor(np.random.default_rng(32).choice(wl.m, q64, replace=False), device=dev)
    qx64 = torch.as_tensor(wl.qx, dtype=torch.float64, device=dev)[i64].contiguous()
    qy64 = torch.as_tensor(wl.qy, dtype=torch.float64, device=dev)[i64].contiguous()
    p64 = aidw.default_params(k=wl.k, levels=wl.levels, precision=aidw.F64)
    ctx.interpolate(ds, qx64, qy64, p64, stream=stream.cuda_stream)
    e0.record(stream)
    ctx.interpolate(ds, qx64, qy64, p64, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    ds.destroy()
    return {"workload": "clustered_2097152_grid_1448x1448", "n": wl.n, "m": wl.m,
            "fp32_ms": ms, "value": wl.n * wl.m / (ms / 1e3), "unit": UNIT,
            "alpha_range": [float(alpha.min()), float(alpha.max())],
            "max_rel_err_vs_fp64_oracle": float(err.max()),
            "max_pure_rel_err_vs_fp64_oracle": float(pure.max()),
            "error_sample": f"{len(idx)} queries (256 seeded, 256 smallest and 256 largest "
                            "alpha) against the oracle on the FP32-rounded inputs",
            "tolerance": 1e-5,
            "fp64_path": {"value": q64 * wl.n / (ms64 / 1e3), "unit": UNIT,
                          "sample": f"{q64} seeded queries x all {wl.n} data points"}}


# ---- GPU arm -----------------------------------------------------------------------------------

def run_batched_leg(args):
    """The batched workload alone (profiling runs of the batch kernel): one JSON line."""
    import torch
    from paper_1511_02186_gb300 import aidw
    import __graft_entry__
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    with aidw.Context(0) as ctx:
        r = bench_batched(ctx, args.steps, args.warmup, dev, torch.cuda.current_stream(dev),
                          tune=args.extras)
    r["note"] = "batched leg alone" + ("" if args.extras else ", built-in kernel shape")
    print(json.dumps(r), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_1511_02186_gb300 import aidw, workloads
    import __graft_entry__
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    __graft_entry__.build()
    job_wl = workloads.uniform_paper(0, n=args.n, m=args.m or args.n)
    wl = rank_workload(job_wl, rank, world, args.scaling)
    # Pair-evaluations of the whole job (all ranks) per step.
    job_pairs = float(job_wl.n) * job_wl.m * (world if args.scaling == "weak" else 1)
    job_queries = job_wl.m * (world if args.scaling == "weak" else 1)
    ctx = aidw.Context(local)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    f64 = args.precision in ("f64", "f64x")
    if f64 and args.extras:
        raise SystemExit(f"--precision {args.precision} is a profiling option: use it with "
                         "--no-extras")
    qdt = torch.float64 if f64 else torch.float32
    qx = torch.as_tensor(wl.qx, dtype=qdt, device=dev)
    qy = torch.as_tensor(wl.qy, dtype=qdt, device=dev)
    out = torch.empty(wl.m, dtype=qdt, device=dev)
    p = aidw.default_params(k=wl.k, levels=wl.levels,
                            precision={"f32": aidw.F32C, "f64": aidw.F64,
                                       "f64x": aidw.F64X}[args.precision])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.interpolate(ds, qx, qy, p, out=out, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ctx.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ktimes = []
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        kt = ctx.kernel_times()  # waits for this step's events
        ktimes.append(kt)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ctx.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, world, dev)
    pairs = float(wl.n) * wl.m  # this rank's
    value = job_pairs * args.steps / total_s

    # Roofline of the dominant kernel (largest device time per step).
    kn = statistics.mean(t.knn_ms for t in ktimes)
    kw = statistics.mean(t.weights_ms for t in ktimes)
    ks = statistics.mean(t.select_ms for t in ktimes)
    kf = statistics.mean(t.finalize_ms for t in ktimes)
    rates = ctx.pipe_rates()
    shape = ctx.tune_config()
    sm = rates.sm_count
    sm_mhz_peak = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_mhz_peak = float(json.load(f).get("sm_max_mhz", sm_mhz_peak))
    except (OSError, ValueError):
        pass
    clk_hz = sm_mhz_peak * 1e6

    def peak_pairs(fp32_ops, mufu_ops):
        # mufu_ops is one lg2 plus one ex2 per pair when nonzero.
        mufu_clk = (1.0 / rates.ex2_per_clk_sm + 1.0 / rates.lg2_per_clk_sm) if mufu_ops else 0.0
        per_pair_clk = max(fp32_ops / LANES_PER_SM, mufu_clk,
                           (fp32_ops + mufu_ops) / LANES_PER_SM)
        return sm * clk_hz / per_pair_clk

    dominant = "weights"
    achieved = pairs / (kw / 1e3)
    peak = peak_pairs(FP32_OPS_P2, MUFU_OPS_P2)
    step_peak = peak
    kernel_sum_s = (kn + kw + ks + kf) / 1e3

    if not args.extras:
        ds.destroy()
        ctx.close()
        if rank == 0:
            metric = {"f32": METRIC, "f64": "AIDW pair-evals/s (FP64 path)",
                      "f64x": "AIDW pair-evals/s (FP64X path)"}[args.precision]
            print(json.dumps({"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "config": workload_config(wl), "precision": args.precision,
                              "kernel_ms": {"knn": kn, "select": ks, "weights": kw,
                                            "finalize": kf},
                              "note": "profiling run without the extra measurements"}))
        return 0

    # FP64 path on a query sample of the same dataset (same per-query work).
    q64 = 8192
    idx = torch.as_tensor(np.random.default_rng(9).choice(wl.m, q64, replace=False))
    qx64 = torch.as_tensor(wl.qx, dtype=torch.float64, device=dev)[idx.to(dev)].contiguous()
    qy64 = torch.as_tensor(wl.qy, dtype=torch.float64, device=dev)[idx.to(dev)].contiguous()
    p64 = aidw.default_params(k=wl.k, levels=wl.levels, precision=aidw.F64)
    ctx.interpolate(ds, qx64, qy64, p64, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.set_profiling(True)
    e0.record(stream)
    ctx.interpolate(ds, qx64, qy64, p64, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    kt64 = ctx.kernel_times()
    ctx.set_profiling(False)
    fp64_rate = q64 * wl.n / (e0.elapsed_time(e1) / 1e3)
    # FP64 phase 2 against the FP64 pipe: FP64 instructions per pair of the kernel as written
    # (distance 4, power scale 1, the weighted sum 1; log2, exp2 and the sum of the weights run
    # in fixed point on the integer pipe) at 2 per clock per SM, GB300's nominal FP64 rate
    # (1.25 TFLOP/s) and the pipe's peak that ncu reports.
    fp64_w_achieved = q64 * wl.n / (kt64.weights_ms / 1e3)
    fp64_w_peak = sm * clk_hz * FP64_PIPE_PER_CLK_SM / FP64_OPS_P2

    # AIDW_F64X (FP64 phase 1 and alpha, double-float phase 2) on a larger query sample, timed
    # the same way; its phase 2 is bound by the four FP64 instructions of each pair's distance.
    q64x = 131072
    idx_x = torch.as_tensor(np.random.default_rng(10).choice(wl.m, q64x, replace=False))
    qx64x = torch.as_tensor(wl.qx, dtype=torch.float64, device=dev)[idx_x.to(dev)].contiguous()
    qy64x = torch.as_tensor(wl.qy, dtype=torch.float64, device=dev)[idx_x.to(dev)].contiguous()
    p64x = aidw.default_params(k=wl.k, levels=wl.levels, precision=aidw.F64X)
    ctx.interpolate(ds, qx64x, qy64x, p64x, stream=stream.cuda_stream)
    ctx.set_profiling(True)
    e0.record(stream)
    ctx.interpolate(ds, qx64x, qy64x, p64x, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    kt64x = ctx.kernel_times()
    ctx.set_profiling(False)
    fp64x_rate = q64x * wl.n / (e0.elapsed_time(e1) / 1e3)
    fp64x_w_achieved = q64x * wl.n / (kt64x.weights_ms / 1e3)
    fp64x_w_peak = sm * clk_hz * FP64_PIPE_PER_CLK_SM / FP64X_OPS_P2

    # End to end through the public API with host buffers: dataset upload (FP64 host arrays),
    # query upload from pinned memory, interpolation, result download.
    hqx = torch.as_tensor(wl.qx, dtype=torch.float32).pin_memory()
    hqy = torch.as_tensor(wl.qy, dtype=torch.float32).pin_memory()
    hout = torch.empty(wl.m, dtype=torch.float32).pin_memory()
    hx, hy, hz = (torch.as_tensor(a, dtype=torch.float64).pin_memory() for a in
                  (wl.x, wl.y, wl.z))
    e2e_steps = max(1, min(args.steps, 3))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d2 = ctx.create_dataset(hx, hy, hz, wl.area)
        ctx.interpolate(d2, hqx, hqy, p, out=hout, stream=stream.cuda_stream)
        d2.destroy()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_val = job_pairs * e2e_steps / e2e_s
    h2d = 3 * 8 * wl.n + 2 * 4 * wl.m
    d2h = 4 * wl.m

    batched = bench_batched(ctx, max(2, args.steps), args.warmup, dev, stream, peak=peak)
    stress = bench_precision_stress(ctx, dev, stream)
    designs = bench_paper_designs(ctx, dev, stream)
    idw = bench_standard_idw(ctx, ds, wl, dev, stream, peak)
    served = None
    if world == 1 or rank == 0:
        sctx = aidw.Context(local)
        # The serving runtime batches many small requests like the batched workload: it runs
        # with the kernel shape the autotuner picked there.
        sctx.set_tune_config(aidw.tune_config(**batched["tuned_config"]))
        served = bench_served(sctx, value / world, args.served_requests, args.nominal_window,
                              args.nominal_queue)
        served["kernel_shape"] = batched["tuned_config"]
        sctx.close()

    line = None
    if rank == 0:
        # The CPU baseline is timed at N = 1 only (with more ranks the host cores are busy
        # feeding the other GPUs): the oracle on all host cores, and on one core (the paper's CPU
        # baseline is serial).
        cpu_v = cpu1_v = None
        if world == 1:
            threads = os.cpu_count() or 1
            cpu_v, cpu_sample, cpu_threads = oracle_rate(wl, args.cpu_seconds, threads)
            cpu1_v, cpu1_sample, _ = oracle_rate(wl, args.cpu_seconds / 3.0, 1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded uniform points in [0,1000]^2, n = m = 1,048,576)",
            "config": dict(workload_config(job_wl), parallelism=(
                "single GPU" if world == 1 else
                f"query sharding over {world} ranks, dataset replicated, no collective on the "
                f"data path ({args.scaling} scaling: " +
                ("each rank its own 1,048,576 queries)" if args.scaling == "weak" else
                 "the workload's queries split into contiguous ranges)"))),
            "queries_per_s": job_queries * args.steps / total_s,
            "kernel_ms": {"knn_incl_query_ordering": kn, "select": ks, "weights": kw,
                          "finalize": kf},
            "plan": {"knn_splits": ktimes[0].splits, "w_splits": ktimes[0].weight_splits,
                     "query_blocks": ktimes[0].query_blocks},
            "roofline": {"bound": "alu",
                         "kernel": (f"f32_{dominant}_kernel<{shape.queries_per_thread}, "
                                    f"{shape.tile_points}>"),
                         "achieved": achieved, "peak": peak, "unit": UNIT,
                         "frac": achieved / peak,
                         "traffic": (measured_traffic(
                             f"f32_weights_kernel<{shape.queries_per_thread}, "
                             f"{shape.tile_points}>") if wl.n == N_DATA and wl.m == M_QUERY
                             else None),
                         "traffic_unit": "bytes per launch (ncu, committed capture)",
                         "peak_basis": (f"{sm} SMs x {sm_mhz_peak:.0f} MHz (max SM clock) / "
                                        "max(7 FP32 ops / 128 lanes, 1/ex2 + 1/lg2 measured MUFU "
                                        "rates per clk per SM, 9 instructions / 128 issue slots)"
                                        " per pair-evaluation of phase 2"),
                         "step_achieved": pairs / kernel_sum_s, "step_peak": step_peak,
                         "step_frac": (pairs / kernel_sum_s) / step_peak,
                         "step_note": "whole step (all kernels incl. query ordering and the "
                                      "pruned phase 1) against the phase-2 bound"},
            "pipe_rates": {"ffma_per_clk_sm": rates.ffma_per_clk_sm,
                           "dfma_per_clk_sm": rates.dfma_per_clk_sm,
                           "ex2_per_clk_sm": rates.ex2_per_clk_sm,
                           "lg2_per_clk_sm": rates.lg2_per_clk_sm,
                           "fmnmx_per_clk_sm": rates.fmnmx_per_clk_sm,
                           "probe_sm_mhz": rates.sm_clock_mhz},
            "fp64_path": {"value": fp64_rate, "unit": UNIT,
                          "sample": f"{q64} seeded queries x all {wl.n} data points",
                          "kernel_ms": {"knn": kt64.knn_ms, "select": kt64.select_ms,
                                        "weights": kt64.weights_ms,
                                        "finalize": kt64.finalize_ms},
                          "roofline": {"bound": "fp64", "kernel": "f64_weights_kernel",
                                       "achieved": fp64_w_achieved, "peak": fp64_w_peak,
                                       "unit": UNIT, "frac": fp64_w_achieved / fp64_w_peak,
                                       "peak_basis": (f"{sm} SMs x {sm_mhz_peak:.0f} MHz x "
                                                      f"{FP64_PIPE_PER_CLK_SM:g} FP64 "
                                                      "instructions per clk per SM (nominal "
                                                      "1.25 TFLOP/s; ncu's FP64 pipe peak) / "
                                                      f"{FP64_OPS_P2} FP64 instructions per "
                                                      "pair"),
                                       "floor_peak": fp64x_w_peak,
                                       "frac_of_floor": fp64_w_achieved / fp64x_w_peak,
                                       "floor_basis": (f"the same FP64 pipe at {FP64X_OPS_P2} "
                                                       "FP64 instructions per pair, the fewest "
                                                       "a pair needs at the FP64 bar as the "
                                                       "FP64X design shows (the squared "
                                                       "distance in FP64, the rest in "
                                                       "double-float on the FP32 pipes)")}},
            "fp64x_path": {"value": fp64x_rate, "unit": UNIT,
                           "sample": f"{q64x} seeded queries x all {wl.n} data points",
                           "kernel_ms": {"knn_incl_query_ordering": kt64x.knn_ms,
                                         "select": kt64x.select_ms,
                                         "weights": kt64x.weights_ms,
                                         "finalize": kt64x.finalize_ms},
                           "roofline": {"bound": "fp64", "kernel": "f64x_weights_kernel",
                                        "achieved": fp64x_w_achieved, "peak": fp64x_w_peak,
                                        "unit": UNIT, "frac": fp64x_w_achieved / fp64x_w_peak,
                                        "peak_basis": (f"{sm} SMs x {sm_mhz_peak:.0f} MHz x "
                                                       f"{FP64_PIPE_PER_CLK_SM:g} FP64 "
                                                       "instructions per clk per SM / "
                                                       f"{FP64X_OPS_P2} FP64 instructions "
                                                       "per pair (the squared distance; "
                                                       "log2, the power, exp2 and the sums "
                                                       "run in double-float on the FP32 "
                                                       "pipes)")}},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "includes": "dataset upload + conversion, query upload, both phases, "
                                "result download"},
            "batched": batched,
            "precision_stress": stress,
            "paper_kernel_designs": designs,
            "standard_idw": idw,
            "served": served,
            "gpu_launches": sum(t.launches for t in ktimes),
            "clocks": clk,
            "cpu_baseline": None if cpu_v is None else {
                "value": cpu_v, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                "sample": cpu_sample},
            "cpu_single_core": None if cpu1_v is None else {
                "value": cpu1_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": cpu1_sample},
            "paper_context": {"gt730m_tiled_soa_1000K_pair_evals_s": 6.2e9,
                              "speedups_over_serial_cpu": {"fp32_naive": 270, "fp32_tiled": 400,
                                                           "fp64": 8},
                              "this_build_over_cpu_oracle": None if cpu_v is None else {
                                  "fp32": value / cpu_v, "fp64": fp64_rate / cpu_v,
                                  "fp64x": fp64x_rate / cpu_v},
                              "this_build_over_single_core_oracle":
                                  None if cpu1_v is None else {
                                      "fp32": value / cpu1_v, "fp64": fp64_rate / cpu1_v},
                              "note": "paper: GeForce GT 730M vs one core of an Intel Core "
                                      "i7-4700MQ, N = 1,024,000, transfers included; here: "
                                      "GB300 vs the FP64 oracle on all host cores; different "
                                      "hardware, baselines and workload"},
        }
    ds.destroy()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=N_DATA,
                    help="data and query count (smaller sizes only for profiling runs)")
    ap.add_argument("--nominal-window", type=float, default=10.0,
                    help="arrival window (s) of the served run at the nominal 2,000 req/s (an "
                         "offered load several times the capacity; refused requests are shed)")
    ap.add_argument("--nominal-queue", type=int, default=64,
                    help="serving queue length during the nominal-rate run")
    ap.add_argument("--served-requests", type=int, default=1000,
                    help="requests offered at each sub-capacity load level of the served run")
    ap.add_argument("--m", type=int, default=0,
                    help="query count (default: --n; smaller sizes only for profiling runs)")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f64x"],
                    help="path of the timed step (f64 and f64x only with --no-extras, for "
                         "profiling)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the FP64, end-to-end and CPU-baseline measurements")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="with N > 1 ranks: weak = every rank its own full query set; strong = "
                         "the workload's queries split over the ranks")
    ap.add_argument("--leg", default="all", choices=["all", "batched"],
                    help="batched: the 256-dataset batched workload alone, for profiling the "
                         "batch kernel (with --no-extras: built-in shape, no autotuning)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg == "batched":
        return run_batched_leg(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
