"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on seeded inputs.

FP32 path: Z within 1e-5 relative to max(|Z*|, S*), kNN sets equal up to FP32 distance ties.
FP64 path: Z within 1e-12, kNN lists bit-identical (same order, ties to the lower index).
FP64X path (FP64 phase 1, double-float phase 2): the FP64 path's bar.
"""
import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import (TOL_F32, TOL_F64, assert_parity, is_f64, knn_mismatch, oracle_for,
                    params_of, rel_err, run_gpu, to_device)

pytestmark = pytest.mark.gpu

PRECISIONS = [aidw.F32C, aidw.F64, aidw.F64X]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = aidw.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_uniform_unit_square_1024(ctx, precision):
    """1,024 data x 1,024 queries uniform in the unit square, A = 1, k = 10."""
    assert_parity(ctx, workloads.uniform_unit(0), precision)


CASES = [
    # (seed, n, m, k, pattern) -- several tiles, ragged tails, k around the list sizes
    (1, 1, 1, 1, "uniform"),
    (2, 7, 33, 7, "uniform"),
    (3, 2047, 129, 10, "clustered"),
    (4, 2049, 515, 8, "uniform"),
    (5, 5000, 777, 9, "clustered"),
    (6, 12345, 3001, 15, "clustered"),
    (7, 4096, 1000, 16, "uniform"),
    (8, 3000, 600, 17, "clustered"),
    (9, 9000, 1500, 32, "clustered"),
    (10, 33, 257, 33 - 1, "uniform"),
]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[1]}m{c[2]}k{c[3]}{c[4][0]}")
def test_small_cases(ctx, precision, case):
    seed, n, m, k, pat = case
    wl = workloads.small_case(seed, n, m, k=k, pattern=pat)
    assert_parity(ctx, wl, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("splits", [(2, 3), (5, 7), (7, 1), (1, 6)])
def test_forced_splits_merge(ctx, precision, splits):
    """Data-range splits restart the neighbour lists and partial sums; merges must agree."""
    wl = workloads.small_case(21, 14000, 900, k=12, pattern="clustered")
    assert_parity(ctx, wl, precision, splits=splits)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_alpha_covers_every_level(ctx, precision):
    """Clustered data with k = 10 spans R from clustered to dispersed (all Eq. 6 segments),
    with non-monotone levels and R_min > 0 (Eq. 5 read with pi / R_max)."""
    wl = workloads.small_case(31, 20000, 2000, k=10, pattern="clustered",
                              levels=(0.7, 2.5, 1.2, 4.0, 3.1))
    wl.r_min, wl.r_max = 0.2, 2.2
    assert_parity(ctx, wl, precision)
    ref, _ = oracle_for(wl, precision)
    segs = np.digitize(ref["alpha"], [0.7 + 1e-9])
    assert len(np.unique(np.round(ref["alpha"], 6))) > 50, "alpha should spread over levels"
    del segs


@pytest.mark.parametrize("precision", PRECISIONS)
def test_equal_levels_is_standard_idw(ctx, precision):
    wl = workloads.small_case(41, 3000, 400, k=5, pattern="clustered", levels=(2.0,) * 5)
    assert_parity(ctx, wl, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_coincident_and_duplicate_points(ctx, precision):
    """Queries on data points, duplicated data points and collinear ties."""
    wl = workloads.small_case(51, 500, 200, k=6, pattern="uniform")
    x, y, z = wl.x.copy(), wl.y.copy(), wl.z.copy()
    x[10:20], y[10:20] = x[0], y[0]          # ten duplicates of point 0
    x[100], y[100] = x[99], y[99]
    wl.x, wl.y = x, y
    qx, qy = wl.qx.copy(), wl.qy.copy()
    qx[:5], qy[:5] = x[[0, 99, 300, 301, 499]], y[[0, 99, 300, 301, 499]]
    wl.qx, wl.qy = qx, qy
    z_gpu, a, kn = run_gpu(ctx, wl, precision)
    assert_parity(ctx, wl, precision, gpu=(z_gpu, a, kn))
    src = wl.as_f32() if precision == aidw.F32C else wl
    expect0 = np.mean(np.concatenate([[src.z[0]], src.z[10:20]]))
    assert abs(z_gpu[0] - expect0) <= 1e-6 * max(1, abs(expect0))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_lattice_ties(ctx, precision):
    """Integer lattice data: many exactly equal distances; kNN ties go to the lower index."""
    rng = np.random.default_rng(61)
    g = np.arange(40, dtype=float)
    gx, gy = np.meshgrid(g, g)
    perm = rng.permutation(1600)
    wl = workloads.Workload("lattice", gx.ravel()[perm], gy.ravel()[perm],
                            rng.standard_normal(1600), 1600.0,
                            rng.integers(0, 80, 300) / 2.0, rng.integers(0, 80, 300) / 2.0, k=9)
    assert_parity(ctx, wl, precision)


def test_host_arrays_match_device_arrays(ctx):
    wl = workloads.small_case(71, 6000, 1234, k=10, pattern="clustered")
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    p = params_of(wl, aidw.F32C)
    zh, ah, kh = ctx.interpolate(ds, wl.qx.astype(np.float32), wl.qy.astype(np.float32), p,
                                 want_alpha=True, want_knn=True)
    zd, ad, kd = run_gpu(ctx, wl, aidw.F32C, ds=ds)
    assert np.array_equal(zh.astype(np.float64), zd)
    assert np.array_equal(kh, kd)
    ds.destroy()


def test_deterministic(ctx):
    wl = workloads.small_case(81, 30000, 5000, k=10, pattern="clustered")
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    a = run_gpu(ctx, wl, aidw.F32C, ds=ds)
    b = run_gpu(ctx, wl, aidw.F32C, ds=ds)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    ds.destroy()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_standard_idw_entry_point(ctx, precision):
    import oracle
    import torch
    wl = workloads.small_case(91, 7000, 800, pattern="clustered")
    src = wl.as_f32() if precision == aidw.F32C else wl
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, precision)
    for p in (1.0, 2.0, 3.5):
        out = ctx.idw(ds, qx, qy, p, precision)
        torch.cuda.synchronize()
        ref = oracle.idw(src.x, src.y, src.z, src.qx, src.qy, p)
        err = rel_err(out.cpu().numpy(), ref)
        assert err.max() <= (TOL_F32 if precision == aidw.F32C else 1e-12)
    ds.destroy()


def test_paper_scale_uniform_sampled(ctx):
    """1,048,576 x 1,048,576 uniform in [0,1000]^2 at the benchmark's launch configuration;
    4,096 sampled queries against the oracle, every output checked for its invariants."""
    wl = workloads.uniform_paper(0)
    z, a, kn = run_gpu(ctx, wl, aidw.F32C, want_knn=False)
    assert np.all(np.isfinite(z))
    zf = wl.as_f32().z
    assert z.min() >= zf.min() - 1e-5 and z.max() <= zf.max() + 1e-5
    assert a.min() >= 1.0 - 1e-6 and a.max() <= 5.0 + 1e-6
    idx = np.random.default_rng(5).choice(wl.m, 4096, replace=False)
    ref, src = oracle_for(wl, aidw.F32C, idx)
    err = rel_err(z[idx], ref)
    assert err.max() <= TOL_F32, err.max()
    assert np.abs(a[idx] - ref["alpha"]).max() <= 1e-5
    # The same launch with the kNN output (the pruned phase 1 keeps indices beside the
    # distances): identical Z and alpha, and the sampled lists equal the oracle's up to FP32
    # distance ties.
    z2, a2, kn = run_gpu(ctx, wl, aidw.F32C, want_knn=True)
    assert np.array_equal(z2, z) and np.array_equal(a2, a)
    bad = knn_mismatch(kn[idx], ref, src, aidw.F32C)
    assert not bad, f"kNN differs beyond ties at sampled queries {bad[:10]}"


def test_clustered_grid_sampled(ctx):
    """2,097,152 clustered data points x 1448^2 grid queries, z lognormal: alpha spans every
    level; 2,048 sampled queries (half random, half the most clustered) against the oracle."""
    wl = workloads.clustered_grid(0)
    z, a, _ = run_gpu(ctx, wl, aidw.F32C, want_knn=False)
    assert np.all(np.isfinite(z)) and np.all(z > 0)
    rng = np.random.default_rng(6)
    idx = np.unique(np.concatenate([rng.choice(wl.m, 1024, replace=False),
                                    np.argsort(a)[:1024]]))
    ref, _ = oracle_for(wl, aidw.F32C, idx)
    err = np.abs(z[idx] - ref["z"]) / np.abs(ref["z"])   # z > 0: pure relative error
    assert err.max() <= TOL_F32, err.max()
    assert ref["alpha"].min() < 1.5 and ref["alpha"].max() > 4.5


@pytest.mark.parametrize("precision", [aidw.F64, aidw.F64X])
def test_fp64_paper_scale_sampled_queries(ctx, precision):
    """FP64 paths on the full 1,048,576-point dataset for 4,096 queries: Z within 1e-12 and
    kNN lists bit-identical."""
    wl = workloads.uniform_paper(0)
    idx = np.random.default_rng(7).choice(wl.m, 4096, replace=False)
    sub = wl.query_subset(idx)
    assert_parity(ctx, sub, precision)


def test_fp64x_paper_scale_launch_sampled(ctx):
    """AIDW_F64X at the benchmark's launch configuration (131,072 queries against the full
    1,048,576-point dataset: Z-ordered queries, pruned phase 1, split phase 2); 1,024 sampled
    queries against the oracle, every output finite and inside the range of z."""
    import torch
    wl = workloads.uniform_paper(0)
    qi = np.random.default_rng(8).choice(wl.m, 131072, replace=False)
    sub = wl.query_subset(qi)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(sub, aidw.F64X)
    out, a, _ = ctx.interpolate(ds, qx, qy, params_of(sub, aidw.F64X), want_alpha=True)
    torch.cuda.synchronize()
    z = out.cpu().numpy()
    assert np.all(np.isfinite(z)) and z.min() >= wl.z.min() and z.max() <= wl.z.max()
    idx = np.random.default_rng(9).choice(sub.m, 1024, replace=False)
    ref, _ = oracle_for(sub, aidw.F64X, idx)
    assert rel_err(z[idx], ref).max() <= TOL_F64
    assert np.abs(a.cpu().numpy()[idx] - ref["alpha"]).max() <= 1e-6
    ds.destroy()


# ---- argument and failure handling on the device ---------------------------------------------

def test_invalid_arguments(ctx):
    wl = workloads.small_case(101, 100, 10)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F32C)
    for bad in (dict(k=0), dict(k=101), dict(k=33), dict(levels=(1, 2, float("nan"), 4, 5)),
                dict(r_min=2.0, r_max=1.0), dict(levels=(1, 2, -3, 4, 5))):
        kw = dict(k=5)
        kw.update(bad)
        with pytest.raises(aidw.AidwError) as e:
            ctx.interpolate(ds, qx, qy, aidw.default_params(**kw))
        assert e.value.status == aidw.ERR_INVALID_ARG
    bad_q = wl.qx.astype(np.float32)
    bad_q[3] = np.inf
    with pytest.raises(aidw.AidwError):
        ctx.interpolate(ds, bad_q, wl.qy.astype(np.float32), aidw.default_params(k=5))
    ds.destroy()
    with pytest.raises(aidw.AidwError) as e:
        ctx.interpolate(ds, qx, qy, aidw.default_params(k=5))
    assert e.value.status == aidw.ERR_INVALID_ARG or e.value.status == aidw.ERR_NOT_FOUND
    x = wl.x.copy()
    x[7] = np.nan
    with pytest.raises(aidw.AidwError) as e:
        ctx.create_dataset(x, wl.y, wl.z, wl.area)
    assert e.value.status == aidw.ERR_INVALID_ARG
    with pytest.raises(aidw.AidwError):
        ctx.create_dataset(wl.x, wl.y, wl.z, 0.0)


def test_budget_and_injected_allocation_failure(ctx):
    wl = workloads.small_case(111, 5000, 500)
    small = aidw.Context(0, hbm_budget=64 << 10)
    with pytest.raises(aidw.AidwError) as e:
        small.create_dataset(wl.x, wl.y, wl.z, wl.area)
    assert e.value.status == aidw.ERR_OOM
    small.close()
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    ctx.fail_alloc_after(0)
    qx, qy = to_device(wl, aidw.F32C)
    with pytest.raises(aidw.AidwError) as e:
        ctx.interpolate(ds, qx, qy, aidw.default_params())
    assert e.value.status == aidw.ERR_OOM
    out, _, _ = ctx.interpolate(ds, qx, qy, aidw.default_params())  # recovers
    assert np.all(np.isfinite(out.cpu().numpy()))
    ds.destroy()


def _fp64_cases():
    rng = np.random.default_rng(91)
    # Enough queries (in FP64, m > 2 x block size x sqrt(resident blocks)) for the pruned phase 1.
    cases = [workloads.small_case(92, 30011, 16411, k=10, pattern="uniform", side=800.0),
             workloads.small_case(93, 50000, 16384, k=17, pattern="clustered", side=300.0),
             workloads.small_case(94, 20000, 9000, k=32, pattern="clustered", side=50.0)]
    # Integer lattice (exact ties everywhere), queries on half-integers and on points.
    g = np.arange(60, dtype=float)
    gx, gy = np.meshgrid(g, g)
    perm = rng.permutation(3600)
    qx = rng.integers(0, 120, 16384) / 2.0
    qy = rng.integers(0, 120, 16384) / 2.0
    cases.append(workloads.Workload("lattice64", gx.ravel()[perm], gy.ravel()[perm],
                                    rng.standard_normal(3600), 3600.0, qx, qy, k=9))
    # Large coordinates with small spacing: FP32 rounding moves points by up to 1/16, far more
    # than their spacing, so the FP32 tile boxes alone would not bound the FP64 distances.
    x = 1.0e6 + rng.uniform(0, 40, 30000)
    y = -2.0e6 + rng.uniform(0, 40, 30000)
    cases.append(workloads.Workload("offset", x, y, rng.standard_normal(30000), 1600.0,
                                    1.0e6 + rng.uniform(0, 40, 16384),
                                    -2.0e6 + rng.uniform(0, 40, 16384), k=10))
    return cases


@pytest.mark.parametrize("idx", range(5), ids=["uniform", "clustered_k17", "clustered_k32",
                                               "lattice_ties", "large_offset"])
def test_fp64_pruned_knn_equals_caller_order_scan(ctx, idx):
    """The three FP64 phase-1 scans: the pruned scan over Z-ordered queries, the caller-order
    split scan and one warp per query, each with and without the kNN output (then the lists hold
    the k smallest (distance, caller index) pairs). All give bit-identical alpha and Z and the
    oracle's kNN lists bit for bit (ties to the lower index), and Z within 1e-12 of the oracle;
    the planned route gives the same."""
    import torch
    wl = _fp64_cases()[idx]
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F64)
    p = aidw.default_params(k=wl.k, precision=aidw.F64)
    ctx.set_profiling(True)
    z1, a1, _ = ctx.interpolate(ds, qx, qy, p, want_alpha=True, splits=(-2, 0))
    assert ctx.kernel_times().launches == 18  # ordering + pruned phase 1
    z2, a2, kn2 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True, splits=(-2, 0))
    assert ctx.kernel_times().launches == 18
    z3, a3, kn3 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True, splits=(4, 0))
    t3 = ctx.kernel_times()
    assert t3.launches == 4 and t3.query_blocks > 0  # caller-order scan
    z4, a4, kn4 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True,
                                  splits=(-1, 0))
    t4 = ctx.kernel_times()
    assert t4.launches == 4 and t4.query_blocks == 0  # one warp per query
    z5, a5, _ = ctx.interpolate(ds, qx, qy, p, want_alpha=True, splits=(-1, 0))
    z0, a0, kn0 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True)
    ctx.set_profiling(False)
    torch.cuda.synchronize()
    for a, z in ((a2, z2), (a3, z3), (a4, z4), (a5, z5), (a0, z0)):
        assert torch.equal(a1, a) and torch.equal(z1, z)
    ref, src = oracle_for(wl, aidw.F64)
    assert rel_err(z1.cpu().numpy(), ref).max() <= TOL_F64
    for kn in (kn2, kn3, kn4, kn0):
        assert np.array_equal(kn.cpu().numpy(), ref["knn"])
    ds.destroy()


@pytest.mark.parametrize("case", [(111, 1_000_000, 300, 10, "uniform"),
                                  (112, 60000, 2000, 32, "clustered"),
                                  (113, 4096, 777, 1, "uniform"),
                                  (114, 2049, 5000, 7, "clustered")],
                         ids=["1M_300q", "clustered_k32", "k1", "ragged_2049"])
def test_fp64_warp_knn_few_queries(ctx, case):
    """FP64 and FP64X calls with few queries against datasets from 2,049 points (padding tiles
    with empty boxes) to 1M, k from 1 to 32: the one-warp-per-query phase 1 gives the oracle's
    kNN lists bit for bit, alpha within 2e-6 of the maximum level and Z within 1e-12; alpha
    and Z equal the caller-order scan's bit for bit."""
    import torch
    seed, n, m, k, pat = case
    wl = workloads.small_case(seed, n, m, k=k, pattern=pat, side=600.0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F64)
    ref, src = oracle_for(wl, aidw.F64)
    for prec in (aidw.F64, aidw.F64X):
        p = params_of(wl, prec)
        ctx.set_profiling(True)
        z1, a1, k1 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True,
                                     splits=(-1, 0))
        assert ctx.kernel_times().query_blocks == 0
        z2, a2, _ = ctx.interpolate(ds, qx, qy, p, want_alpha=True, splits=(3, 0))
        ctx.set_profiling(False)
        torch.cuda.synchronize()
        assert torch.equal(a1, a2) and torch.equal(z1, z2)
        assert np.array_equal(k1.cpu().numpy(), ref["knn"])
        assert np.abs(a1.cpu().numpy() - ref["alpha"]).max() <= 2e-6 * 5.0
        assert rel_err(z1.cpu().numpy(), ref).max() <= TOL_F64
    ds.destroy()


@pytest.mark.parametrize("idx", range(5), ids=["uniform", "clustered_k17", "clustered_k32",
                                               "lattice_ties", "large_offset"])
def test_fp64x_matches_fp64_path(ctx, idx):
    """AIDW_F64X shares the FP64 path's phase 1 and selection: alpha and the kNN lists are
    bit-identical to AIDW_F64's; Z differs only by the double-float phase 2, within 1e-13 of
    the FP64 path, and both within 1e-12 of the oracle."""
    import torch
    wl = _fp64_cases()[idx]
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F64)
    z64, a64, k64 = ctx.interpolate(ds, qx, qy, params_of(wl, aidw.F64), want_alpha=True,
                                    want_knn=True)
    zx, ax, kx = ctx.interpolate(ds, qx, qy, params_of(wl, aidw.F64X), want_alpha=True,
                                 want_knn=True)
    zs, _, _ = ctx.interpolate(ds, qx, qy, params_of(wl, aidw.F64X), splits=(3, 5))
    torch.cuda.synchronize()
    assert torch.equal(a64, ax) and torch.equal(k64, kx)
    ref, _ = oracle_for(wl, aidw.F64)
    for z in (z64, zx, zs):
        assert rel_err(z.cpu().numpy(), ref).max() <= TOL_F64
    den = np.maximum(np.abs(z64.cpu().numpy()), ref["scale"])
    assert (np.abs(zx.cpu().numpy() - z64.cpu().numpy()) / den).max() <= 1e-13
    ds.destroy()


def test_fp64x_extreme_powers(ctx):
    """Levels up to 40 (weights falling as d^-40 span far more than the float exponent range:
    the ones below 2^-126 of the nearest point's are dropped) and down to 0.05 (nearly equal
    weights over the whole dataset): the FP64 bar still holds."""
    wl = workloads.small_case(98, 20000, 3000, k=10, pattern="clustered", side=400.0,
                              levels=(0.05, 1.0, 8.0, 20.0, 40.0))
    assert_parity(ctx, wl, aidw.F64X)
    ref, _ = oracle_for(wl, aidw.F64X)
    assert ref["alpha"].min() < 0.5 and ref["alpha"].max() > 30.0


@pytest.mark.parametrize("pattern", ["uniform", "clustered"])
def test_fp32_pruned_knn_equals_split_scan(ctx, pattern):
    """FP32 with enough queries for the pruned phase 1 (more than 32,768) against the forced
    split scan: kNN lists equal to the oracle's up to FP32 distance ties, alpha within FP32
    rounding, both Z within tolerance of the oracle."""
    import torch
    wl = workloads.small_case(95, 30000, 60000, k=10, pattern=pattern, side=500.0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F32C)
    p = params_of(wl, aidw.F32C)
    ctx.set_profiling(True)
    z1, a1, k1 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True)
    assert ctx.kernel_times().launches == 18  # ordering + pruned phase 1
    z2, a2, k2 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True, splits=(8, 0))
    assert ctx.kernel_times().launches == 4
    ctx.set_profiling(False)
    torch.cuda.synchronize()
    ref, src = oracle_for(wl, aidw.F32C)
    for z in (z1, z2):
        assert rel_err(z.cpu().numpy(), ref).max() <= TOL_F32
    # Both scans' lists against the oracle's, element by element: a differing index must tie
    # the oracle's k-th distance within FP32 rounding.
    for kn in (k1, k2):
        bad = knn_mismatch(kn.cpu().numpy(), ref, src, aidw.F32C)
        assert not bad, f"kNN differs beyond ties at queries {bad[:10]}"
    assert np.abs(a1.cpu().numpy() - a2.cpu().numpy()).max() <= 1e-5
    ds.destroy()


@pytest.mark.parametrize("case", [(96, 60000, 20000, 10, "clustered"),
                                  (97, 1000000 // 8, 3000, 32, "uniform"),
                                  (98, 5000, 32768, 7, "clustered"),
                                  (99, 4096, 100, 1, "uniform")],
                         ids=lambda c: f"n{c[1]}m{c[2]}k{c[3]}{c[4][0]}")
def test_fp32_warp_knn_matches_the_block_scans(ctx, case):
    """Up to 32,768 queries the FP32 path finds each query's neighbours with one warp per query
    (box hierarchy, bitonic merges across the lanes). Its k smallest distances are those of the
    block scans, so alpha and Z are bit-identical to the forced split scan's with the same
    phase-2 plan, and the lists equal the oracle's up to FP32 distance ties."""
    import torch
    seed, n, m, k, pat = case
    wl = workloads.small_case(seed, n, m, k=k, pattern=pat, side=400.0)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F32C)
    p = params_of(wl, aidw.F32C)
    ctx.set_profiling(True)
    z1, a1, k1 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True)
    t1 = ctx.kernel_times()
    assert t1.launches == 4 and t1.query_blocks == 0  # one warp per query
    z2, a2, k2 = ctx.interpolate(ds, qx, qy, p, want_alpha=True, want_knn=True,
                                 splits=(3, t1.weight_splits))
    assert ctx.kernel_times().splits > 1  # a split scan (at most one split per 2,048 points)
    ctx.set_profiling(False)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(z1, z2)
    ref, src = oracle_for(wl, aidw.F32C)
    assert rel_err(z1.cpu().numpy(), ref).max() <= TOL_F32
    bad = knn_mismatch(k1.cpu().numpy(), ref, src, aidw.F32C)
    assert not bad, f"kNN differs beyond ties at queries {bad[:10]}"
    ds.destroy()


def _degenerate_cases():
    rng = np.random.default_rng(97)
    out = []
    # Every data point at one location (zero-area bounding box), queries around and on it.
    x = np.full(3000, 12.5)
    y = np.full(3000, -3.0)
    qx = np.concatenate([[12.5], rng.uniform(0, 25, 2999)])
    qy = np.concatenate([[-3.0], rng.uniform(-15, 9, 2999)])
    out.append(workloads.Workload("one_location", x, y, rng.standard_normal(3000), 600.0,
                                  qx, qy, k=10))
    # k = n (every point is a neighbour).
    x, y = rng.uniform(0, 1, 12), rng.uniform(0, 1, 12)
    out.append(workloads.Workload("k_equals_n", x, y, rng.standard_normal(12), 1.0,
                                  rng.uniform(0, 1, 300), rng.uniform(0, 1, 300), k=12))
    # Collinear data (zero width in y), queries off the line.
    x = rng.uniform(0, 100, 5000)
    out.append(workloads.Workload("collinear", x, np.zeros(5000), np.sin(x), 100.0,
                                  rng.uniform(0, 100, 2500), rng.uniform(-5, 5, 2500), k=8))
    # Two dense clusters 1e4 apart: weights span hundreds of decades.
    x = np.concatenate([rng.normal(0, 0.01, 2000), rng.normal(1e4, 0.01, 2000)])
    y = np.concatenate([rng.normal(0, 0.01, 2000), rng.normal(0, 0.01, 2000)])
    z = np.concatenate([np.ones(2000), -np.ones(2000)]) + 0.01 * rng.standard_normal(4000)
    out.append(workloads.Workload("two_clusters", x, y, z, 1e8,
                                  rng.uniform(-1, 1e4 + 1, 2500), rng.uniform(-1, 1, 2500),
                                  k=10))
    # Large coordinate offset with small spacing (FP32 coordinates near 1e5).
    x = 1.0e5 + rng.uniform(0, 50, 8000)
    y = 2.0e5 + rng.uniform(0, 50, 8000)
    out.append(workloads.Workload("offset_1e5", x, y, np.cos(x / 7), 2500.0,
                                  1.0e5 + rng.uniform(0, 50, 3000),
                                  2.0e5 + rng.uniform(0, 50, 3000), k=10))
    # Queries far outside the data's box (every data point far and at nearly the same
    # distance: R large, alpha at the top level, the weights nearly equal).
    x, y = rng.uniform(0, 1, 6000), rng.uniform(0, 1, 6000)
    out.append(workloads.Workload("far_queries", x, y, np.sin(7 * x) * y, 1.0,
                                  rng.uniform(300, 301, 2000), rng.uniform(-301, -300, 2000),
                                  k=10))
    return out


# Phase-1 routes a test can force (one warp per query, the pruned scan over Z-ordered queries,
# the split scan with three data splits), each with the same phase-2 plan (two data splits).
ROUTES = {"warp": (-1, 2), "pruned": (-2, 2), "split3": (3, 2)}


DEGENERATE_IDS = ["one_location", "k_equals_n", "collinear", "two_clusters", "offset_1e5",
                  "far_queries"]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("idx", range(len(DEGENERATE_IDS)), ids=DEGENERATE_IDS)
def test_degenerate_inputs(ctx, precision, idx):
    """Zero-area and zero-width data, k = n, weights spanning hundreds of decades, large
    coordinate offsets and queries far outside the data: the same parity as the regular
    cases."""
    wl = _degenerate_cases()[idx]
    assert_parity(ctx, wl, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("idx", range(len(DEGENERATE_IDS)), ids=DEGENERATE_IDS)
def test_degenerate_inputs_every_phase1_route(ctx, precision, idx):
    """The degenerate geometries through each phase-1 scan, whatever the sizes would pick: one
    warp per query, the pruned scan (its tile and sub-tile boxes of zero width or area, a query
    block's box far from every tile) and the split scan. Each route meets the oracle's bar (Z,
    alpha, kNN lists up to FP32 ties; FP64 lists bit for bit), and alpha and Z agree between
    the routes bit for bit (they keep the same k smallest distances)."""
    wl = _degenerate_cases()[idx]
    runs = {}
    for name, splits in ROUTES.items():
        runs[name] = run_gpu(ctx, wl, precision, want_knn=True, splits=splits)
        assert_parity(ctx, wl, precision, gpu=runs[name])
    z0, a0, _ = runs["warp"]
    for name in ("pruned", "split3"):
        z, a, _ = runs[name]
        assert np.array_equal(a, a0), f"{wl.name}: alpha differs between warp and {name}"
        assert np.array_equal(z, z0), f"{wl.name}: Z differs between warp and {name}"


@pytest.mark.parametrize("precision", PRECISIONS)
def test_empty_query_set_and_empty_dataset(ctx, precision):
    """m = 0 is a no-op for every entry point (outputs untouched); n = 0 is rejected."""
    import torch
    wl = workloads.small_case(121, 50, 5, k=3)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    dt = torch.float64 if is_f64(precision) else torch.float32
    e = torch.empty(0, dtype=dt, device="cuda")
    p = aidw.default_params(k=3, precision=precision)
    out, a, kn = ctx.interpolate(ds, e, e, p, want_alpha=True, want_knn=True)
    torch.cuda.synchronize()
    assert out.numel() == 0 and a.numel() == 0 and kn.numel() == 0
    out = ctx.idw(ds, e, e, 2.0, precision=precision)
    assert out.numel() == 0
    h = np.zeros(0, dtype=np.float64 if is_f64(precision) else np.float32)
    out, _, _ = ctx.interpolate(ds, h, h, p)
    assert out.shape == (0,)
    if is_f64(precision):
        rc, rid = ctx.submit(ds, h, h, p, np.zeros(0))
        assert rc == aidw.OK and ctx.wait(rid, 10_000_000) == aidw.OK
        ctx.release(rid)
    ds.destroy()
    with pytest.raises(aidw.AidwError) as err:
        ctx.create_dataset(np.zeros(0), np.zeros(0), np.zeros(0), 1.0)
    assert err.value.status == aidw.ERR_INVALID_ARG
