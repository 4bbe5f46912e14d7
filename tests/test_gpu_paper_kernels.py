"""The paper's kernel designs (naive / tiled, SoA / AoaS; Sec. 3.1) rebuilt for comparison.

Each of the four variants must match the oracle at the path's tolerance (FP32 1e-5, FP64 1e-12,
alpha included), the four variants of one precision must give identical bits (same arithmetic,
only layout and tiling differ), and the FP64 variants must equal the optimized FP64 path within
its tolerance."""
import itertools

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32, TOL_F64, oracle_for, params_of, rel_err, to_device

pytestmark = pytest.mark.gpu

VARIANTS = list(itertools.product((aidw.VERSION_NAIVE, aidw.VERSION_TILED),
                                  (aidw.LAYOUT_SOA, aidw.LAYOUT_AOAS)))
PRECISIONS = [aidw.F32C, aidw.F64]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = aidw.Context(0)
    yield c
    c.close()


def run_variants(ctx, wl, precision):
    import torch
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, precision)
    res = {}
    for version, layout in VARIANTS:
        out, oa = ctx.interpolate_paper(ds, qx, qy, params_of(wl, precision), version=version,
                                        layout=layout, want_alpha=True)
        torch.cuda.synchronize()
        res[(version, layout)] = (out.cpu().numpy().astype(np.float64), oa.cpu().numpy())
    ds.destroy()
    return res


def check(ctx, wl, precision):
    res = run_variants(ctx, wl, precision)
    ref, _ = oracle_for(wl, precision)
    tol = TOL_F64 if precision == aidw.F64 else TOL_F32
    base = res[VARIANTS[0]]
    for v, (z, a) in res.items():
        assert rel_err(z, ref).max() <= tol, (v, rel_err(z, ref).max())
        atol = 1e-12 if precision == aidw.F64 else 2e-6
        assert np.abs(a - ref["alpha"]).max() <= atol * max(wl.levels) + 1e-6, v
        assert np.array_equal(z, base[0]) and np.array_equal(a, base[1]), v
    return res


CASES = [
    dict(seed=1, n=3001, m=777, k=10, pattern="uniform"),
    dict(seed=2, n=5000, m=1000, k=17, pattern="clustered"),
    dict(seed=3, n=257, m=300, k=32, pattern="uniform"),
    dict(seed=4, n=1, m=5, k=1, pattern="uniform"),
    dict(seed=5, n=2048, m=256, k=8, pattern="clustered"),
]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['pattern']}_{c['n']}x{c['m']}_k{c['k']}")
def test_variants_match_oracle_and_each_other(ctx, precision, case):
    c = dict(case)
    wl = workloads.small_case(c.pop("seed"), c.pop("n"), c.pop("m"), k=c.pop("k"),
                              pattern=c.pop("pattern"), side=200.0)
    check(ctx, wl, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_coincident_queries_and_duplicates(ctx, precision):
    wl = workloads.small_case(6, 700, 120, k=6, pattern="uniform")
    x, y = wl.x.copy(), wl.y.copy()
    x[10:20], y[10:20] = x[0], y[0]
    wl.x, wl.y = x, y
    qx, qy = wl.qx.copy(), wl.qy.copy()
    qx[:3], qy[:3] = x[[0, 5, 699]], y[[0, 5, 699]]
    wl.qx, wl.qy = qx, qy
    res = check(ctx, wl, precision)
    src = wl.as_f32() if precision == aidw.F32C else wl
    expect0 = np.mean(np.concatenate([[src.z[0]], src.z[10:20]]))
    z0 = res[VARIANTS[0]][0][0]
    assert abs(z0 - expect0) <= 1e-6 * max(1.0, abs(expect0))


def test_fp64_variants_equal_optimized_path(ctx):
    import torch
    wl = workloads.small_case(7, 4000, 900, k=10, pattern="clustered", side=300.0)
    res = run_variants(ctx, wl, aidw.F64)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F64)
    out, a, _ = ctx.interpolate(ds, qx, qy, params_of(wl, aidw.F64), want_alpha=True)
    torch.cuda.synchronize()
    z_opt = out.cpu().numpy()
    z_pap = res[VARIANTS[0]][0]
    assert np.abs(z_opt - z_pap).max() <= 1e-12 * max(1.0, np.abs(z_opt).max())
    assert np.array_equal(a.cpu().numpy(), res[VARIANTS[0]][1])
    ds.destroy()


def test_rejects_bad_arguments(ctx):
    import torch
    wl = workloads.small_case(8, 100, 10, k=3)
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, aidw.F32C)
    p = params_of(wl, aidw.F32C)
    for version, layout in ((2, 0), (0, 2), (-1, 0)):
        with pytest.raises(aidw.AidwError):
            ctx.interpolate_paper(ds, qx, qy, p, version=version, layout=layout)
    with pytest.raises(aidw.AidwError):  # host arrays are not accepted
        ctx.interpolate_paper(ds, qx.cpu(), qy.cpu(), p, out=torch.empty(10))
    q64 = to_device(wl, aidw.F64)
    with pytest.raises(aidw.AidwError):  # the paper's designs have no double-float variant
        ctx.interpolate_paper(ds, *q64, params_of(wl, aidw.F64X))
    ds.destroy()
