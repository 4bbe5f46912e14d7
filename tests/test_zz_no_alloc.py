"""The allocation-free entry point, aidw_interpolate_noalloc, called through the C ABI.

It exists for callers that may not allocate device memory while serving a call (a process
with a device footprint fixed at start-up, or code that cannot accept the device
synchronisation of cudaFree). It must give the same predictions as aidw_interpolate, call after
call, although every call reuses one fixed scratch array inside the library.

This file is collected last on purpose, so that a run that stops at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, workloads
from parity import TOL_F32

pytestmark = pytest.mark.gpu


def _noalloc(ctx, ds, qx, qy, params, out):
    import torch
    rc = ctx.lib.aidw_interpolate_noalloc(ctx.ptr, ds.handle, qx.data_ptr(), qy.data_ptr(),
                                          int(qx.shape[0]), ctypes.byref(params),
                                          out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    return rc


def _check_against_interpolate(ctx, wl):
    """One call of each entry point on the same device arrays; predictions within the FP32
    tolerance, relative to max(|Z|, sum w|z| / sum w) (z changes sign)."""
    import torch
    ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
    qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
    qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
    p = aidw.default_params(k=wl.k, levels=wl.levels)
    ref, _, _ = ctx.interpolate(ds, qx, qy, p)
    # Condition scale of each prediction, from the same weights: the denominator the parity
    # tests use.
    ds_abs = ctx.create_dataset(wl.x, wl.y, np.abs(wl.z), wl.area)
    scale_t, _, _ = ctx.interpolate(ds_abs, qx, qy, p)
    out = torch.full((wl.m,), float("nan"), dtype=torch.float32, device="cuda")
    assert _noalloc(ctx, ds, qx, qy, p, out) == aidw.OK
    torch.cuda.synchronize()
    assert ctx.check_device_errors() == aidw.OK
    a = out.cpu().numpy().astype(np.float64)
    b = ref.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a))
    scale = np.maximum(np.abs(b), scale_t.cpu().numpy().astype(np.float64))
    assert (np.abs(a - b) / scale).max() <= TOL_F32
    ds.destroy()
    ds_abs.destroy()


def test_noalloc_matches_interpolate_twice():
    """Two calls in a row on the pruned phase-1 route (more than 32,768 queries, scratch fits),
    different sizes, the same scratch array."""
    import torch
    assert torch.cuda.is_available()
    with aidw.Context(0) as ctx:
        for wl in (workloads.small_case(201, 40000, 60000, k=10, pattern="clustered"),
                   workloads.small_case(202, 25000, 50000, k=15, pattern="uniform")):
            _check_against_interpolate(ctx, wl)


def test_noalloc_other_routes():
    """Fewer queries (one warp per query, as aidw_interpolate) and more queries than the pruned
    route's scratch allows at k = 10 (split scan with fewer splits)."""
    with aidw.Context(0) as ctx:
        for wl in (workloads.small_case(204, 30000, 3000, k=10, pattern="clustered"),
                   workloads.small_case(205, 6000, 230000, k=10, pattern="uniform")):
            _check_against_interpolate(ctx, wl)


def test_noalloc_call_allocates_nothing():
    """After a first call of the same size (under lazy module loading the driver loads kernel
    code at a kernel's first launch), further calls leave the device's free memory unchanged."""
    import torch
    with aidw.Context(0) as ctx:
        wl = workloads.small_case(206, 20000, 40000, k=10, pattern="clustered")
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
        out = torch.empty(wl.m, dtype=torch.float32, device="cuda")
        p = aidw.default_params(k=10)
        assert _noalloc(ctx, ds, qx, qy, p, out) == aidw.OK
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            assert _noalloc(ctx, ds, qx, qy, p, out) == aidw.OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        assert ctx.check_device_errors() == aidw.OK
        ds.destroy()


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    with aidw.Context(0) as ctx:
        wl = workloads.small_case(203, 5000, 300000, k=10)
        ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
        p = aidw.default_params(k=10)
        qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
        qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
        out = torch.empty(wl.m, dtype=torch.float32, device="cuda")
        # 300,000 queries at k = 10 need more than the 16 MiB scratch array.
        assert _noalloc(ctx, ds, qx, qy, p, out) == aidw.ERR_INVALID_ARG
        # Host arrays would need staging buffers, i.e. an allocation.
        hq = np.zeros(10, dtype=np.float32)
        rc = ctx.lib.aidw_interpolate_noalloc(ctx.ptr, ds.handle, hq.ctypes.data,
                                              hq.ctypes.data, 10, ctypes.byref(p),
                                              hq.ctypes.data, None)
        assert rc == aidw.ERR_INVALID_ARG
        for prec in (aidw.F64, aidw.F64X):
            p64 = aidw.default_params(k=10, precision=prec)
            assert _noalloc(ctx, ds, qx[:10], qy[:10], p64, out) == aidw.ERR_INVALID_ARG
        ds.destroy()
