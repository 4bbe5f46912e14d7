"""Parity helpers shared by the GPU tests: run the CUDA path through the C ABI and compare it
with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1511_02186_gb300 import aidw

# Tolerances on Z: max relative error against max(|Z*|, S*), S* = sum(w|z|)/sum(w) the
# condition scale of the weighted mean.
TOL_F32 = 1e-5
TOL_F64 = 1e-12
# kNN index sets of the FP32 path may differ only where a distance ties the k-th one within
# FP32 rounding of the squared distance (a few ulp).
KNN_TIE_REL_F32 = 2e-6


def is_f64(precision):
    """AIDW_F64 and AIDW_F64X take FP64 arrays and share the FP64 parity bar."""
    return precision in (aidw.F64, aidw.F64X)


def oracle_for(wl, precision, q_idx=None, threads=None):
    """Oracle result on the inputs the given path actually sees (FP32-rounded for F32C)."""
    src = wl.as_f32() if precision == aidw.F32C else wl
    if q_idx is not None:
        src = src.query_subset(q_idx)
    return oracle.interpolate(src.x, src.y, src.z, src.area, src.qx, src.qy, src.k, src.levels,
                              src.r_min, src.r_max, threads=threads), src


def rel_err(z, ref):
    den = np.maximum(np.abs(ref["z"]), ref["scale"])
    return np.abs(np.asarray(z, dtype=np.float64) - ref["z"]) / den


def knn_mismatch(knn_gpu, ref, src, precision):
    """Indices of queries whose kNN set differs beyond what ties explain."""
    knn_gpu = np.asarray(knn_gpu, dtype=np.int64)
    bad = []
    for q in range(knn_gpu.shape[0]):
        a, b = knn_gpu[q], ref["knn"][q]
        if is_f64(precision):
            if not np.array_equal(a, b):
                bad.append(q)
            continue
        sa, sb = set(a.tolist()), set(b.tolist())
        if sa == sb:
            continue
        if min(a) < 0 or max(a) >= src.n:
            bad.append(q)
            continue
        dk = (src.qx[q] - src.x[b[-1]]) ** 2 + (src.qy[q] - src.y[b[-1]]) ** 2
        for i in sa ^ sb:
            di = (src.qx[q] - src.x[i]) ** 2 + (src.qy[q] - src.y[i]) ** 2
            if abs(di - dk) > KNN_TIE_REL_F32 * max(dk, 1e-300):
                bad.append(q)
                break
    return bad


def to_device(wl, precision):
    import torch
    dt = torch.float64 if is_f64(precision) else torch.float32
    return (torch.as_tensor(wl.qx, dtype=dt, device="cuda"),
            torch.as_tensor(wl.qy, dtype=dt, device="cuda"))


def params_of(wl, precision):
    return aidw.default_params(k=wl.k, levels=wl.levels, r_min=wl.r_min, r_max=wl.r_max,
                               precision=precision)


def run_gpu(ctx, wl, precision, want_knn=True, splits=None, ds=None):
    """Interpolate on the GPU with device tensors; returns numpy (z, alpha, knn)."""
    import torch
    own = ds is None
    if own:
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx, qy = to_device(wl, precision)
    out, a, kn = ctx.interpolate(ds, qx, qy, params_of(wl, precision), want_alpha=True,
                                 want_knn=want_knn, splits=splits)
    torch.cuda.synchronize()
    res = (out.cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64),
           None if kn is None else kn.cpu().numpy())
    if own:
        ds.destroy()
    return res


def assert_parity(ctx, wl, precision, want_knn=True, splits=None, q_idx=None, gpu=None):
    """Full comparison: Z within tolerance, alpha close, kNN sets equal up to ties."""
    z, a, kn = gpu if gpu is not None else run_gpu(ctx, wl, precision, want_knn, splits)
    ref, src = oracle_for(wl, precision, q_idx)
    if q_idx is not None:
        z, a = z[q_idx], a[q_idx]
        kn = None if kn is None else kn[q_idx]
    tol = TOL_F64 if is_f64(precision) else TOL_F32
    err = rel_err(z, ref)
    assert np.all(np.isfinite(z)), "non-finite prediction"
    worst = int(np.argmax(err))
    assert err.max() <= tol, (f"{wl.name}: max rel err {err.max():.3e} at query {worst} "
                              f"(gpu {z[worst]!r}, oracle {ref['z'][worst]!r})")
    # alpha is returned as float: FP32 rounding for the FP64 path; for the FP32 path also the
    # FP32 rounding of r_obs propagated through Eq. 5-6.
    atol_alpha = (2e-7 if is_f64(precision) else 2e-6) * max(wl.levels)
    if kn is not None:
        bad = knn_mismatch(kn, ref, src, precision)
        assert not bad, f"{wl.name}: kNN differs at queries {bad[:10]}"
        # alpha depends on the kNN multiset of distances only.
        da = np.abs(a - ref["alpha"])
        assert da.max() <= atol_alpha, f"{wl.name}: alpha err {da.max():.3e}"
    return err.max()
