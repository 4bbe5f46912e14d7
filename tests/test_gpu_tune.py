"""Kernel shapes and the autotuner on the GPU.

Every shape field except the batched split length is arithmetic-neutral, so results must be
bit-identical across those fields; every shape must match the oracle within the FP32
tolerance; the autotuners must return a valid shape, leave the winner's results in the outputs
and record / reuse it through the tuning cache.
"""
import json

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32, oracle_for, params_of, rel_err, to_device

pytestmark = pytest.mark.gpu

NEUTRAL = [
    dict(queries_per_thread=4, knn_queries_per_thread=0),
    dict(queries_per_thread=4),
    dict(queries_per_thread=8),
    dict(tile_points=256),
    dict(knn_list=16),
    dict(knn_list=32),
    dict(knn_queries_per_thread=2),
    dict(queries_per_thread=8, tile_points=256, knn_list=32, ctas_per_sm=2),
    dict(queries_per_thread=2, knn_queries_per_thread=2, knn_list=16),
    dict(unit_order=1),
]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = aidw.Context(0)
    yield c
    c.close()


@pytest.fixture(autouse=True)
def fresh_cache():
    aidw.TuneCache.clear()
    yield
    aidw.TuneCache.clear()


def interp(ctx, ds, wl, cfg, splits=None):
    import torch
    ctx.set_tune_config(cfg)
    try:
        qx, qy = to_device(wl, aidw.F32C)
        out, a, _ = ctx.interpolate(ds, qx, qy, params_of(wl, aidw.F32C), want_alpha=True,
                                    splits=splits)
        torch.cuda.synchronize()
        assert ctx.check_device_errors() == aidw.OK
        return out.cpu().numpy(), a.cpu().numpy()
    finally:
        ctx.set_tune_config(aidw.tune_config())


def test_single_call_shapes_are_neutral_and_match_oracle(ctx):
    wl = workloads.small_case(71, 30011, 5003, k=10, pattern="clustered", side=500.0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    ref, _ = oracle_for(wl, aidw.F32C)
    # Fixed split counts: only the neutral fields differ, so the bits must not.
    base_z, base_a = interp(ctx, ds, wl, aidw.tune_config(), splits=(2, 3))
    for f in NEUTRAL:
        z, a = interp(ctx, ds, wl, aidw.tune_config(**f), splits=(2, 3))
        assert np.array_equal(z, base_z), f
        assert np.array_equal(a, base_a), f
    # Planned splits (and the pruned phase 1): each shape within tolerance of the oracle.
    for f in [{}] + NEUTRAL:
        z, _ = interp(ctx, ds, wl, aidw.tune_config(**f))
        assert rel_err(z, ref).max() <= TOL_F32, f
    ds.destroy()


def make_items(ctx, wls):
    import torch
    items = []
    for wl in wls:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx, qy = to_device(wl, aidw.F32C)
        out = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
        items.append((ds, qx, qy, params_of(wl, aidw.F32C), out, None))
    return items


def batch_workloads(seed):
    rng = np.random.default_rng(seed)
    wls = []
    for i in range(7):
        n = int(np.exp(rng.uniform(np.log(500), np.log(150000))))
        m = int(np.exp(rng.uniform(np.log(100), np.log(20000))))
        k = int(rng.choice([6, 10, 15]))
        wls.append(workloads.small_case(seed * 100 + i, n, m, k=k,
                                        pattern="clustered" if i % 2 else "uniform",
                                        side=float(rng.uniform(10, 1000))))
    return wls


def outputs(items):
    import torch
    torch.cuda.synchronize()
    return [it[4].cpu().numpy().copy() for it in items]


def test_batch_shapes_neutral_and_split_length_within_tolerance(ctx):
    wls = batch_workloads(5)
    items = make_items(ctx, wls)
    pb = ctx.batch_create(items)
    assert pb.config() == aidw.tune_config()
    pb.launch()
    base = outputs(items)
    refs = [oracle_for(wl, aidw.F32C)[0] for wl in wls]
    for z, ref in zip(base, refs):
        assert rel_err(z, ref).max() <= TOL_F32
    for f in NEUTRAL:
        cfg = aidw.tune_config(**f)
        pb.set_config(cfg)
        assert pb.config() == cfg
        for it in items:
            it[4].fill_(float("nan"))
        pb.launch()
        for z, b in zip(outputs(items), base):
            assert np.array_equal(z, b), f
    for sp in (2048, 16384, 262144):
        pb.set_config(aidw.tune_config(split_points=sp))
        pb.launch()
        for z, ref in zip(outputs(items), refs):
            assert rel_err(z, ref).max() <= TOL_F32, sp
    assert ctx.check_device_errors() == aidw.OK
    with pytest.raises(aidw.AidwError):
        pb.set_config(aidw.tune_config(tile_points=1000))
    # A rejected shape leaves the batch as it was.
    pb.launch()
    assert all(rel_err(z, ref).max() <= TOL_F32 for z, ref in zip(outputs(items), refs))
    pb.destroy()
    for it in items:
        it[0].destroy()


def test_batch_autotune_and_cache(ctx, tmp_path):
    wls = batch_workloads(6)
    items = make_items(ctx, wls)
    pb = ctx.batch_create(items)
    for it in items:
        it[4].fill_(float("nan"))
    cfg, ms = pb.autotune(reps=2, flags=aidw.TUNE_CACHE)
    assert aidw.tune_config_valid(cfg) and ms > 0
    assert pb.config() == cfg
    refs = [oracle_for(wl, aidw.F32C)[0] for wl in wls]
    for z, ref in zip(outputs(items), refs):
        assert rel_err(z, ref).max() <= TOL_F32
    assert aidw.TuneCache.size() == 1
    path = tmp_path / "tune.jsonl"
    aidw.TuneCache.save(str(path))
    (obj,) = [json.loads(l) for l in path.read_text().splitlines() if l.strip()]
    assert obj["key"].startswith("batch dev=sm_")
    assert {f: obj[f] for f in aidw.TuneConfig.FIELDS} == cfg.as_dict()
    # A cache hit reuses the stored shape without timing, also in a fresh batch.
    aidw.TuneCache.clear()
    assert aidw.TuneCache.load(str(path)) == aidw.OK
    pb2 = ctx.batch_create(items)
    cfg2, ms2 = pb2.autotune(reps=2, flags=aidw.TUNE_CACHE)
    assert cfg2 == cfg and ms2 == -1.0 and pb2.config() == cfg
    pb2.launch()
    for z, ref in zip(outputs(items), refs):
        assert rel_err(z, ref).max() <= TOL_F32
    pb2.destroy()
    pb.destroy()
    for it in items:
        it[0].destroy()


def test_autotune_interpolate_applies_and_caches(ctx):
    import torch
    wl = workloads.small_case(72, 60000, 20000, k=10, pattern="uniform", side=1000.0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F32C)
    p = params_of(wl, aidw.F32C)
    try:
        cfg, ms, out = ctx.autotune_interpolate(ds, qx, qy, p, reps=2,
                                                flags=aidw.TUNE_CACHE | aidw.TUNE_APPLY)
        torch.cuda.synchronize()
        assert aidw.tune_config_valid(cfg) and ms > 0
        assert ctx.tune_config() == cfg
        ref, _ = oracle_for(wl, aidw.F32C)
        assert rel_err(out.cpu().numpy(), ref).max() <= TOL_F32
        out.fill_(float("nan"))
        cfg2, ms2, out2 = ctx.autotune_interpolate(ds, qx, qy, p, out=out, reps=2,
                                                   flags=aidw.TUNE_CACHE)
        torch.cuda.synchronize()
        assert cfg2 == cfg and ms2 == -1.0
        assert rel_err(out2.cpu().numpy(), ref).max() <= TOL_F32
        with pytest.raises(aidw.AidwError):
            ctx.autotune_interpolate(ds, qx.cpu(), qy.cpu(), p, out=out.cpu())
    finally:
        ctx.set_tune_config(aidw.tune_config())
        ds.destroy()


def test_serving_keeps_the_shape_it_started_with():
    import torch
    with aidw.Context(0) as c:
        c.set_tune_config(aidw.tune_config(queries_per_thread=2, split_points=16384))
        wl = workloads.small_case(73, 20000, 3000, k=10, pattern="clustered", side=300.0)
        ds = c.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx, qy = to_device(wl, aidw.F32C)
        out1 = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
        rc, r1 = c.submit(ds, qx, qy, params_of(wl, aidw.F32C), out1)
        assert rc == aidw.OK and c.wait(r1, 60_000_000) == aidw.OK
        c.set_tune_config(aidw.tune_config())
        out2 = torch.full_like(out1, float("nan"))
        rc, r2 = c.submit(ds, qx, qy, params_of(wl, aidw.F32C), out2)
        assert rc == aidw.OK and c.wait(r2, 60_000_000) == aidw.OK
        torch.cuda.synchronize()
        assert torch.equal(out1, out2)
        ref, _ = oracle_for(wl, aidw.F32C)
        assert rel_err(out1.cpu().numpy(), ref).max() <= TOL_F32
