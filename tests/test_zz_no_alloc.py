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


def test_noalloc_matches_interpolate_twice():
    import torch
    assert torch.cuda.is_available()
    with aidw.Context(0) as ctx:
        runs = [workloads.small_case(201, 40000, 30000, k=10, pattern="clustered"),
                workloads.small_case(202, 25000, 50000, k=15, pattern="uniform")]
        for wl in runs:  # two calls in a row, different sizes, same scratch array
            ds = ctx.create_dataset(wl.x, wl.y, wl.z, wl.area)
            qx = torch.as_tensor(wl.qx, dtype=torch.float32, device="cuda")
            qy = torch.as_tensor(wl.qy, dtype=torch.float32, device="cuda")
            p = aidw.default_params(k=wl.k, levels=wl.levels)
            ref, _, _ = ctx.interpolate(ds, qx, qy, p)
            # Condition scale sum(w|z|)/sum(w) of each prediction, from the same weights: the
            # denominator the parity tests use, since z changes sign.
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
