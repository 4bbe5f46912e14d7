"""Batched interpolation (one persistent work-queue kernel for many datasets) on the GPU.

Checks every item against the FP64 oracle, that an item's result is bit-identical alone and in
any mix (the work split depends only on the item), and the prepared, graph-replayed batch.
"""
import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32, oracle_for, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = aidw.Context(0)
    yield c
    c.close()


def make_items(ctx, wls):
    import torch
    items, keep = [], []
    for wl in wls:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
        out = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
        oa = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
        p = aidw.default_params(k=wl.k, levels=wl.levels, r_min=wl.r_min, r_max=wl.r_max)
        items.append((ds, qx, qy, p, out, oa))
        keep.append(wl)
    return items


def mixed_workloads(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1, 40000))
        m = int(rng.integers(1, 9000))
        k = int(rng.choice([1, 6, 10, 15, 20, 32]))
        k = min(k, n)
        pat = "clustered" if rng.uniform() < 0.5 else "uniform"
        side = float(np.exp(rng.uniform(np.log(10), np.log(1000))))
        levels = tuple(np.round(rng.uniform(0.5, 6.0, 5), 3))
        out.append(workloads.small_case(seed * 1000 + i, n, m, k=k, pattern=pat, side=side,
                                        levels=levels))
    return out


def test_batch_items_match_oracle(ctx):
    import torch
    wls = mixed_workloads(1, 12)
    items = make_items(ctx, wls)
    ctx.interpolate_batch(items)
    torch.cuda.synchronize()
    assert ctx.check_device_errors() == aidw.OK
    for wl, (ds, qx, qy, p, out, oa) in zip(wls, items):
        z = out.cpu().numpy().astype(np.float64)
        ref, _ = oracle_for(wl, aidw.F32C)
        err = rel_err(z, ref)
        assert err.max() <= TOL_F32, (wl.name, wl.k, err.max())
        da = np.abs(oa.cpu().numpy() - ref["alpha"]).max()
        assert da <= 2e-6 * max(wl.levels), (wl.name, da)
    for it in items:
        it[0].destroy()


def test_alone_equals_in_mix_bitwise(ctx):
    import torch
    wls = mixed_workloads(2, 9)
    items = make_items(ctx, wls)
    ctx.interpolate_batch(items)
    torch.cuda.synchronize()
    mixed = [it[4].clone() for it in items]
    for i in (0, 4, 8):
        ds, qx, qy, p, out, oa = items[i]
        out.fill_(float("nan"))
        ctx.interpolate_batch([items[i]])
        torch.cuda.synchronize()
        assert torch.equal(out, mixed[i]), f"item {i} differs alone vs in the mix"
    # A different mix (reversed, with duplicates of one dataset) gives the same bits again.
    rev = list(reversed(items)) + [items[3]]
    for it in rev:
        it[4].fill_(float("nan"))
    ctx.interpolate_batch(rev)
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        assert torch.equal(it[4], mixed[i])
    for it in items:
        it[0].destroy()


def test_batch_matches_single_call(ctx):
    import torch
    wls = mixed_workloads(3, 5)
    items = make_items(ctx, wls)
    ctx.interpolate_batch(items)
    torch.cuda.synchronize()
    for wl, (ds, qx, qy, p, out, oa) in zip(wls, items):
        single, _, _ = ctx.interpolate(ds, qx, qy, p)
        torch.cuda.synchronize()
        ref, _ = oracle_for(wl, aidw.F32C)
        # Both within tolerance of the oracle, and of each other on its scale.
        a, b = out.cpu().numpy().astype(np.float64), single.cpu().numpy().astype(np.float64)
        den = np.maximum(np.abs(ref["z"]), ref["scale"])
        assert (np.abs(a - b) / den).max() <= 2 * TOL_F32
    for it in items:
        it[0].destroy()


def test_prepared_batch_graph_replay(ctx):
    import torch
    wls = mixed_workloads(4, 6)
    items = make_items(ctx, wls)
    pb = ctx.batch_create(items)
    pb.launch()
    torch.cuda.synchronize()
    first = [it[4].clone() for it in items]
    for it in items:
        it[4].fill_(float("nan"))
    pb.launch()
    torch.cuda.synchronize()
    for i, it in enumerate(items):
        assert torch.equal(it[4], first[i])
    # Rewrite one item's queries in place: the replay picks up the new contents.
    wl = wls[2]
    ds, qx, qy, p, out, oa = items[2]
    rng = np.random.default_rng(9)
    side = np.sqrt(wl.area)
    newx, newy = rng.uniform(0, side, wl.m), rng.uniform(0, side, wl.m)
    qx.copy_(torch.as_tensor(newx, dtype=torch.float32))
    qy.copy_(torch.as_tensor(newy, dtype=torch.float32))
    pb.launch()
    torch.cuda.synchronize()
    wl2 = workloads.Workload("moved", wl.x, wl.y, wl.z, wl.area, newx, newy, k=wl.k,
                             levels=wl.levels)
    ref, _ = oracle_for(wl2, aidw.F32C)
    assert rel_err(out.cpu().numpy(), ref).max() <= TOL_F32
    pb.destroy()
    for it in items:
        it[0].destroy()


def test_batch_edge_cases(ctx):
    import torch
    ctx.interpolate_batch([])
    wl = workloads.small_case(5, 100, 10, k=3)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    empty = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.interpolate_batch([(ds, empty, empty, aidw.default_params(k=3), empty, None)])
    qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
    with pytest.raises(aidw.AidwError):  # host output array
        ctx.interpolate_batch([(ds, qx, qx, aidw.default_params(k=3),
                                torch.empty(10, dtype=torch.float32), None)])
    for prec in (aidw.F64, aidw.F64X):  # only the FP32 path is batched
        with pytest.raises(aidw.AidwError):
            ctx.interpolate_batch([(ds, qx, qx, aidw.default_params(k=3, precision=prec),
                                    torch.empty(10, dtype=torch.float32, device="cuda"), None)])
    ds.destroy()


def test_full_size_batched_workload_sampled(ctx):
    """The benchmark's 256-dataset batch, prepared and autotuned as bench.py times it: 16
    seeded queries of every item against the oracle (every query of small items is still in the
    batch), plus the invariants on all outputs (finite, within [min z, max z])."""
    import torch
    wls = workloads.batched(0)
    items = []
    for wl in wls:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
        out = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
        items.append((ds, qx, qy, aidw.default_params(k=wl.k), out, None))
    pb = ctx.batch_create(items)
    pb.autotune(reps=1)
    for it in items:
        it[4].fill_(float("nan"))
    pb.launch()
    torch.cuda.synchronize()
    assert ctx.check_device_errors() == aidw.OK
    rng = np.random.default_rng(77)
    worst = 0.0
    for wl, it in zip(wls, items):
        z = it[4].cpu().numpy().astype(np.float64)
        src = wl.as_f32()
        assert np.isfinite(z).all()
        assert z.min() >= src.z.min() - 1e-5 and z.max() <= src.z.max() + 1e-5
        idx = rng.choice(wl.m, 16, replace=False)
        ref, _ = oracle_for(wl, aidw.F32C, q_idx=idx)
        worst = max(worst, rel_err(z[idx], ref).max())
    assert worst <= TOL_F32, worst
    pb.destroy()
    for it in items:
        it[0].destroy()
