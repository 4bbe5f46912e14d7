"""Serving with continuous batching (aidw_submit / aidw_poll / aidw_wait) on the GPU.

Requests of different datasets and sizes are admitted by device footprint into persistent batch
launches that overlap on two streams; each result must equal the oracle within tolerance and be
bit-identical to the same request served alone.
"""
import time

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32, TOL_F64, oracle_for, rel_err

pytestmark = pytest.mark.gpu


def datasets(ctx, seed, count, n_max=60000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(64, n_max))
        wl = workloads.small_case(seed * 100 + i, n, 1, k=10,
                                  pattern="clustered" if i % 2 else "uniform",
                                  side=float(rng.uniform(10, 1000)))
        out.append((wl, ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)))
    return out


def request(wl, seed, m, device):
    import torch
    rng = np.random.default_rng(seed)
    side = np.sqrt(wl.area)
    qx, qy = rng.uniform(0, side, m), rng.uniform(0, side, m)
    w = workloads.Workload(wl.name, wl.x, wl.y, wl.z, wl.area, qx, qy, k=wl.k)
    if device:
        tq = (torch.as_tensor(qx, dtype=torch.float32, device="cuda"),
              torch.as_tensor(qy, dtype=torch.float32, device="cuda"))
        out = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
    else:
        tq = (qx.astype(np.float32), qy.astype(np.float32))
        out = np.full(m, np.nan, dtype=np.float32)
    return w, tq, out


def to_np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else a


def test_served_requests_match_oracle_and_overlap():
    with aidw.Context(0) as ctx:
        dss = datasets(ctx, 1, 6)
        rng = np.random.default_rng(2)
        reqs = []
        for i in range(40):
            wl, ds = dss[int(rng.integers(0, len(dss)))]
            m = int(rng.integers(1, 6000))
            w, (qx, qy), out = request(wl, 1000 + i, m, device=bool(i % 2))
            p = aidw.default_params(k=10)
            rc, rid = ctx.submit(ds, qx, qy, p, out)
            assert rc == aidw.OK
            reqs.append((w, rid, out, (qx, qy)))
        for w, rid, out, _ in reqs:
            assert ctx.wait(rid, 60_000_000) == aidw.OK
        for w, rid, out, _ in reqs:
            ref, _ = oracle_for(w, aidw.F32C)
            assert rel_err(to_np(out), ref).max() <= TOL_F32
            assert ctx.latency_us(rid) > 0
            assert ctx.release(rid) == aidw.OK
        st = ctx.serving_stats()
        assert st.completed == 40 and st.failed == 0
        assert st.batched_requests == 40
        assert st.launches < 40, "requests should share launches"
        assert st.max_concurrent_launches >= 2, "launches should overlap on the device"


def test_alone_equals_in_the_mix():
    import torch
    with aidw.Context(0) as ctx:
        dss = datasets(ctx, 3, 4)
        wl, ds = dss[1]
        w, (qx, qy), out_alone = request(wl, 77, 4321, device=True)
        p = aidw.default_params(k=10)
        rc, rid = ctx.submit(ds, qx, qy, p, out_alone)
        assert rc == aidw.OK and ctx.wait(rid, 60_000_000) == aidw.OK
        # The same request again, submitted inside a burst of others.
        out_mix = torch.full_like(out_alone, float("nan"))
        ids = []
        for i in range(12):
            wl2, ds2 = dss[i % 4]
            _, (a, b), o = request(wl2, 500 + i, 1000 + 300 * i, device=True)
            ids.append((ctx.submit(ds2, a, b, p, o)[1], (a, b, o)))
            if i == 6:
                rc, mid = ctx.submit(ds, qx, qy, p, out_mix)
                assert rc == aidw.OK
        for rid2, _ in ids:
            assert ctx.wait(rid2, 60_000_000) == aidw.OK
        assert ctx.wait(mid, 60_000_000) == aidw.OK
        torch.cuda.synchronize()
        assert torch.equal(out_alone, out_mix)


def test_admission_by_footprint_and_oversize():
    with aidw.Context(0) as ctx:
        ctx.serving_configure(inflight_bytes=6 << 20, max_batch_requests=4, streams=2)
        dss = datasets(ctx, 4, 3, n_max=20000)
        p = aidw.default_params(k=10)
        reqs = []
        for i in range(16):
            wl, ds = dss[i % 3]
            w, (qx, qy), out = request(wl, 900 + i, 3000, device=False)
            rc, rid = ctx.submit(ds, qx, qy, p, out)
            assert rc == aidw.OK
            reqs.append((w, rid, out))
        for w, rid, out in reqs:
            assert ctx.wait(rid, 60_000_000) == aidw.OK
            ref, _ = oracle_for(w, aidw.F32C)
            assert rel_err(out, ref).max() <= TOL_F32
        st = ctx.serving_stats()
        assert st.launches >= 4  # at most 4 requests per launch
        assert st.in_flight_bytes == 0
        # A request whose footprint alone exceeds the budget fails with OOM, not a hang.
        wl, ds = dss[0]
        w, (qx, qy), out = request(wl, 1, 200000, device=False)
        rc, rid = ctx.submit(ds, qx, qy, p, out)
        assert rc == aidw.OK
        assert ctx.wait(rid, 60_000_000) == aidw.ERR_OOM


def test_solo_paths_fp64_and_knn():
    import torch
    with aidw.Context(0) as ctx:
        dss = datasets(ctx, 5, 2)
        wl, ds = dss[0]
        rng = np.random.default_rng(8)
        side = np.sqrt(wl.area)
        qx, qy = rng.uniform(0, side, 700), rng.uniform(0, side, 700)
        w = workloads.Workload(wl.name, wl.x, wl.y, wl.z, wl.area, qx, qy, k=10)
        out64 = np.full(700, np.nan)
        p64 = aidw.default_params(k=10, precision=aidw.F64)
        rc, r1 = ctx.submit(ds, qx, qy, p64, out64)
        assert rc == aidw.OK
        out64x = np.full(700, np.nan)
        rc, r3 = ctx.submit(ds, qx, qy, aidw.default_params(k=10, precision=aidw.F64X), out64x)
        assert rc == aidw.OK
        out32 = np.full(700, np.nan, dtype=np.float32)
        knn = np.full((700, 10), -1, dtype=np.int32)
        rc, r2 = ctx.submit(ds, qx.astype(np.float32), qy.astype(np.float32),
                            aidw.default_params(k=10), out32, out_knn=knn)
        assert rc == aidw.OK
        assert ctx.wait(r1, 60_000_000) == aidw.OK and ctx.wait(r2, 60_000_000) == aidw.OK
        ref64, _ = oracle_for(w, aidw.F64)
        assert rel_err(out64, ref64).max() <= TOL_F64
        assert ctx.wait(r3, 60_000_000) == aidw.OK
        assert rel_err(out64x, ref64).max() <= TOL_F64
        ref32, _ = oracle_for(w, aidw.F32C)
        assert rel_err(out32, ref32).max() <= TOL_F32
        assert (knn >= 0).all()
        rc, done = ctx.poll(r1)
        assert rc == aidw.OK and done
        assert ctx.release(r1) == aidw.OK
        assert ctx.poll(r1)[0] == aidw.ERR_NOT_FOUND
        del torch


def test_submit_rejects_bad_requests():
    with aidw.Context(0) as ctx:
        wl = workloads.small_case(9, 50, 5, k=3)
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        out = np.zeros(5, dtype=np.float32)
        q = wl.qx.astype(np.float32)
        assert ctx.submit(ds, q, q, aidw.default_params(k=51), out)[0] == aidw.ERR_INVALID_ARG
        bad = q.copy()
        bad[2] = np.nan
        assert ctx.submit(ds, bad, q, aidw.default_params(k=3), out)[0] == aidw.ERR_INVALID_ARG
        ds.destroy()
        assert ctx.submit(ds, q, q, aidw.default_params(k=3), out)[0] in (
            aidw.ERR_NOT_FOUND, aidw.ERR_INVALID_ARG)
        time.sleep(0.01)


def test_full_size_served_workload_sampled():
    """Requests of the benchmark's served workload (64 resident datasets of 16K-1M points,
    256-262,144 host-array queries each), submitted as a burst: 16 seeded queries of each of
    the first 24 requests against the oracle, and every output finite."""
    with aidw.Context(0) as ctx:
        dsw = workloads.served_datasets(0)
        handles = [ctx.create_dataset(w.x, w.y, w.z, w.area) for w in dsw]
        p = aidw.default_params(k=10)
        reqs = workloads.served_requests(dsw, seed=12, rate=200.0, duration_s=1.0)[:24]
        subs = []
        for _, d, qx, qy in reqs:
            out = np.full(len(qx), np.nan, dtype=np.float32)
            q32x, q32y = qx.astype(np.float32), qy.astype(np.float32)
            rc, rid = ctx.submit(handles[d], q32x, q32y, p, out)
            assert rc == aidw.OK
            subs.append((d, qx, qy, out, rid))
        rng = np.random.default_rng(5)
        worst = 0.0
        for d, qx, qy, out, rid in subs:
            assert ctx.wait(rid, 120_000_000) == aidw.OK
            assert np.isfinite(out).all()
            w = dsw[d]
            wl = workloads.Workload(w.name, w.x, w.y, w.z, w.area, qx, qy, k=10)
            idx = rng.choice(len(qx), min(16, len(qx)), replace=False)
            ref, _ = oracle_for(wl, aidw.F32C, q_idx=idx)
            worst = max(worst, rel_err(out[idx], ref).max())
            ctx.release(rid)
        assert worst <= TOL_F32, worst
        st = ctx.serving_stats()
        assert st.completed == len(subs) and st.failed == 0


def test_backpressure_queue_full_then_resubmit():
    """A queue of 3 requests served one request per launch on one stream: a burst of submits
    overfills it, aidw_submit refuses with AIDW_ERR_AGAIN (nothing accepted, counted in the
    stats) and the client resubmits after a pause; every request then completes and matches the
    oracle. A longer limit set while the runtime is running takes the next burst whole."""
    with aidw.Context(0) as ctx:
        ctx.serving_configure(max_batch_requests=1, streams=1, max_queued=3)
        dss = datasets(ctx, 6, 2, n_max=20000)
        p = aidw.default_params(k=10)
        reqs = [request(dss[i % 2][0], 1200 + i, 3000, device=False) + (dss[i % 2][1],)
                for i in range(24)]
        accepted, again = [], 0
        for w, (qx, qy), out, ds in reqs:
            while True:
                rc, rid = ctx.submit(ds, qx, qy, p, out)
                if rc != aidw.ERR_AGAIN:
                    break
                assert rid == 0
                again += 1
                time.sleep(0.0005)
            assert rc == aidw.OK
            accepted.append((w, rid, out))
        assert again >= 1, "a burst of 24 should overfill a queue of 3"
        for w, rid, out in accepted:
            assert ctx.wait(rid, 60_000_000) == aidw.OK
            ref, _ = oracle_for(w, aidw.F32C)
            assert rel_err(out, ref).max() <= TOL_F32
            assert ctx.release(rid) == aidw.OK
        st = ctx.serving_stats()
        assert st.rejected_again == again
        assert st.completed == 24 and st.failed == 0 and st.queued == 0
        # A longer queue, set while the runtime runs: the same burst is taken without refusal.
        ctx.serving_set_queue_limit(64)
        ids = []
        for w, (qx, qy), out, ds in reqs:
            rc, rid = ctx.submit(ds, qx, qy, p, out)
            assert rc == aidw.OK
            ids.append(rid)
        for rid in ids:
            assert ctx.wait(rid, 60_000_000) == aidw.OK
        assert ctx.serving_stats().rejected_again == again
        with pytest.raises(aidw.AidwError):
            ctx.serving_set_queue_limit(0)


def test_large_request_served_in_chunks():
    """A request of 250,000 queries against 400,000 points (1e11 pair-evaluations) is cut into
    three chunks of whole query blocks served by separate launches, and a small request
    submitted after it rides in one of the first launches, so it completes first. The large
    request's result matches the oracle on sampled queries and is bit-identical to the same
    request served alone (the cut depends on its own sizes only)."""
    import torch
    with aidw.Context(0) as ctx:
        big = workloads.small_case(61, 400000, 250000, k=10, pattern="clustered", side=800.0)
        ds = ctx.create_dataset(big.x, big.y, big.z, big.area)
        small = workloads.small_case(62, 5000, 2000, k=10, pattern="uniform", side=800.0)
        ds2 = ctx.create_dataset(small.x, small.y, small.z, small.area)
        p = aidw.default_params(k=10)
        qx = torch.as_tensor(big.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(big.qy, dtype=torch.float32, device="cuda")
        out_alone = torch.full((big.m,), float("nan"), dtype=torch.float32, device="cuda")
        rc, rid = ctx.submit(ds, qx, qy, p, out_alone)
        assert rc == aidw.OK and ctx.wait(rid, 120_000_000) == aidw.OK
        launches0 = ctx.serving_stats().launches
        assert launches0 >= 3, "the large request should take three launches"
        out_mix = torch.full_like(out_alone, float("nan"))
        sq = small.qx.astype(np.float32), small.qy.astype(np.float32)
        out_small = np.full(small.m, np.nan, dtype=np.float32)
        rc, rbig = ctx.submit(ds, qx, qy, p, out_mix)
        rc2, rsmall = ctx.submit(ds2, sq[0], sq[1], p, out_small)
        assert rc == aidw.OK and rc2 == aidw.OK
        assert ctx.wait(rbig, 120_000_000) == aidw.OK and ctx.wait(rsmall, 60_000_000) == aidw.OK
        assert ctx.latency_us(rsmall) < ctx.latency_us(rbig)
        torch.cuda.synchronize()
        assert torch.equal(out_alone, out_mix)
        idx = np.random.default_rng(3).choice(big.m, 512, replace=False)
        ref, _ = oracle_for(big, aidw.F32C, q_idx=idx)
        assert rel_err(out_mix.cpu().numpy()[idx], ref).max() <= TOL_F32
        ref_s, _ = oracle_for(small, aidw.F32C)
        assert rel_err(out_small, ref_s).max() <= TOL_F32
        # The same request from host arrays with the alpha output: every chunk is staged and
        # written back at its own offset.
        hx, hy = big.qx.astype(np.float32), big.qy.astype(np.float32)
        hout = np.full(big.m, np.nan, dtype=np.float32)
        halpha = np.full(big.m, np.nan, dtype=np.float32)
        rc, rh = ctx.submit(ds, hx, hy, p, hout, out_alpha=halpha)
        assert rc == aidw.OK and ctx.wait(rh, 120_000_000) == aidw.OK
        assert np.array_equal(hout, out_alone.cpu().numpy())
        assert np.all(np.isfinite(halpha))
        assert np.abs(halpha[idx] - ref["alpha"]).max() <= 1e-5
