"""Python binding of ``libaidw.so`` (the C ABI in ``include/aidw.h``).

Argument marshalling only: every step of the interpolation runs in the library's CUDA kernels.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA memory); torch provides
device memory and streams, nothing else. If the compiled library is missing this module raises
instead of falling back to any other implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libaidw.so")

OK = 0
PENDING = 1
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_AGAIN = -3
ERR_TIMEOUT = -4
ERR_CUDA = -5
ERR_NOT_FOUND = -6
ERR_UNSUPPORTED = -7

F32C = 0
F64 = 1
F64X = 2
DTYPE_F32 = 0
DTYPE_F64 = 1
MAX_K = 32
VERSION_NAIVE = 0
VERSION_TILED = 1
LAYOUT_SOA = 0
LAYOUT_AOAS = 1

_lock = threading.Lock()
_lib = None


class AidwError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class Params(ctypes.Structure):
    """``aidw_params``: k, precision, alpha levels (Eq. 6), R_min / R_max (Eq. 5)."""
    _fields_ = [("k", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("alpha", ctypes.c_double * 5), ("r_min", ctypes.c_double),
                ("r_max", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_int32)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("knn_ms", ctypes.c_double), ("select_ms", ctypes.c_double),
                ("weights_ms", ctypes.c_double), ("finalize_ms", ctypes.c_double),
                ("splits", ctypes.c_int32), ("query_blocks", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("weight_splits", ctypes.c_int32)]


class PipeRates(ctypes.Structure):
    _fields_ = [("ffma_per_clk_sm", ctypes.c_double), ("ex2_per_clk_sm", ctypes.c_double),
                ("lg2_per_clk_sm", ctypes.c_double), ("fmnmx_per_clk_sm", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sm_count", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dfma_per_clk_sm", ctypes.c_double)]


class ServingStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("rejected_again", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("max_concurrent_launches", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("queued", ctypes.c_int64), ("in_flight_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t)]


class BatchItem(ctypes.Structure):
    _fields_ = [("ds", ctypes.c_int64), ("qx", ctypes.c_void_p), ("qy", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("params", Params), ("out", ctypes.c_void_p),
                ("out_alpha", ctypes.c_void_p)]


class TuneConfig(ctypes.Structure):
    """``aidw_tune_config``: kernel shape (phase-2 queries per thread and tile points, k-list
    length, points per batched phase-2 unit, persistent CTAs per SM, phase-1 queries per
    thread, batch unit order)."""
    _fields_ = [("queries_per_thread", ctypes.c_int32), ("tile_points", ctypes.c_int32),
                ("knn_list", ctypes.c_int32), ("split_points", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("knn_queries_per_thread", ctypes.c_int32),
                ("unit_order", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    FIELDS = ("queries_per_thread", "tile_points", "knn_list", "split_points", "ctas_per_sm",
              "knn_queries_per_thread", "unit_order")

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f in self.FIELDS}

    def __eq__(self, other):
        return isinstance(other, TuneConfig) and self.as_dict() == other.as_dict()

    def __repr__(self):
        return f"TuneConfig({self.as_dict()})"


TUNE_CACHE = 1
TUNE_APPLY = 2


# Every symbol of include/aidw.h with its signature (restype, argtypes).
_P, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "aidw_params_default": (None, [_P]),
    "aidw_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_size_t]),
    "aidw_shutdown": (ctypes.c_int, [_P]),
    "aidw_create_dataset": (ctypes.c_int, [_P, _P, _P, _P, _I64, _D, _I32, _P]),
    "aidw_destroy_dataset": (ctypes.c_int, [_P, _I64]),
    "aidw_dataset_info": (ctypes.c_int, [_P, _I64, _P, _P]),
    "aidw_interpolate": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "aidw_idw": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _D, _I32, _P, _P]),
    "aidw_interpolate_noalloc": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P]),
    "aidw_interpolate_batch": (ctypes.c_int, [_P, _P, _I32, _P]),
    "aidw_batch_create": (ctypes.c_int, [_P, _P, _I32, _P]),
    "aidw_batch_launch": (ctypes.c_int, [_P, _P, _P]),
    "aidw_batch_destroy": (ctypes.c_int, [_P, _P]),
    "aidw_submit": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "aidw_poll": (ctypes.c_int, [_P, _I64, _P]),
    "aidw_wait": (ctypes.c_int, [_P, _I64, _I64]),
    "aidw_request_latency_us": (ctypes.c_int, [_P, _I64, _P]),
    "aidw_release_request": (ctypes.c_int, [_P, _I64]),
    "aidw_serving_configure": (ctypes.c_int, [_P, ctypes.c_size_t, _I32, _I32, _I64]),
    "aidw_serving_set_queue_limit": (ctypes.c_int, [_P, _I64]),
    "aidw_serving_get_stats": (ctypes.c_int, [_P, _P]),
    "aidw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "aidw_check_device_errors": (ctypes.c_int, [_P]),
    "aidw_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "aidw_last_kernel_times": (ctypes.c_int, [_P, _P]),
    "aidw_measure_pipe_rates": (ctypes.c_int, [_P, _P]),
    "aidw_debug_fail_alloc_after": (ctypes.c_int, [_P, _I64]),
    "aidw_debug_expire_wait": (ctypes.c_int, [_P, _I32, ctypes.c_uint32]),
    "aidw_interpolate_paper": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _I32, _I32,
                                              _P]),
    "aidw_tune_config_default": (ctypes.c_int, [_P]),
    "aidw_tune_config_check": (ctypes.c_int, [_P]),
    "aidw_set_tune_config": (ctypes.c_int, [_P, _P]),
    "aidw_get_tune_config": (ctypes.c_int, [_P, _P]),
    "aidw_autotune_interpolate": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _I32,
                                                 ctypes.c_uint32, _P, _P]),
    "aidw_batch_set_config": (ctypes.c_int, [_P, _P, _P]),
    "aidw_batch_get_config": (ctypes.c_int, [_P, _P, _P]),
    "aidw_batch_autotune": (ctypes.c_int, [_P, _P, _I32, ctypes.c_uint32, _P, _P]),
    "aidw_tune_cache_put": (ctypes.c_int, [ctypes.c_char_p, _P, _D]),
    "aidw_tune_cache_get": (ctypes.c_int, [ctypes.c_char_p, _P, _P]),
    "aidw_tune_cache_clear": (ctypes.c_int, []),
    "aidw_tune_cache_size": (ctypes.c_int, []),
    "aidw_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "aidw_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "aidw_debug_f64_log2_exp2": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "aidw_debug_df_weight": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P]),
}
# Test-only hooks exported by the library but not declared in the public header.
DEBUG_SIGNATURES = {
    "aidw_debug_admission": (ctypes.c_int, [_I64, _P, _P, ctypes.c_uint64, ctypes.c_uint64, _I32,
                                            _P, _D, _P]),
    "aidw_debug_interpolate_splits": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P,
                                                     _I32, _I32]),
}


def load(path: str = LIB_PATH):
    """Load libaidw.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in {**SIGNATURES, **DEBUG_SIGNATURES}.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().aidw_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise AidwError(rc, what)


def default_params(k: int = 10, levels=(1.0, 2.0, 3.0, 4.0, 5.0), r_min: float = 0.0,
                   r_max: float = 2.0, precision: int = F32C) -> Params:
    p = Params()
    load().aidw_params_default(ctypes.byref(p))
    p.k = int(k)
    p.precision = int(precision)
    for i, a in enumerate(levels):
        p.alpha[i] = float(a)
    p.r_min = float(r_min)
    p.r_max = float(r_max)
    return p


def tune_config(**fields) -> TuneConfig:
    """The built-in kernel shape with the given fields replaced."""
    c = TuneConfig()
    _check(load().aidw_tune_config_default(ctypes.byref(c)), "tune_config_default")
    for k, v in fields.items():
        if k not in TuneConfig.FIELDS:
            raise KeyError(k)
        setattr(c, k, int(v))
    return c


def tune_config_valid(c: TuneConfig) -> bool:
    return load().aidw_tune_config_check(ctypes.byref(c)) == OK


class TuneCache:
    """The library's process-wide tuning cache (host only)."""

    @staticmethod
    def put(key: str, cfg: TuneConfig, ms: float = -1.0):
        _check(load().aidw_tune_cache_put(key.encode(), ctypes.byref(cfg), float(ms)),
               "tune_cache_put")

    @staticmethod
    def get(key: str):
        """(TuneConfig, ms) or None for an unknown key."""
        c, ms = TuneConfig(), ctypes.c_double()
        rc = load().aidw_tune_cache_get(key.encode(), ctypes.byref(c), ctypes.byref(ms))
        if rc == ERR_NOT_FOUND:
            return None
        _check(rc, "tune_cache_get")
        return c, ms.value

    @staticmethod
    def clear():
        _check(load().aidw_tune_cache_clear(), "tune_cache_clear")

    @staticmethod
    def size() -> int:
        return int(load().aidw_tune_cache_size())

    @staticmethod
    def save(path: str):
        _check(load().aidw_tune_cache_save(os.fsencode(path)), "tune_cache_save")

    @staticmethod
    def load(path: str) -> int:
        """Merges a cache file; returns the status (OK, ERR_NOT_FOUND, ERR_INVALID_ARG)."""
        return int(load().aidw_tune_cache_load(os.fsencode(path)))


# ---- array marshalling -------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _prep(a, dtype):
    """Returns (keepalive, pointer) for a 1-D contiguous array of `dtype` ('f4','f8','i4')."""
    if _is_torch(a):
        import torch
        tdt = {"f4": torch.float32, "f8": torch.float64, "i4": torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor, got {a.dtype}")
        return a, a.data_ptr()
    arr = np.asarray(a)
    if arr.dtype != np.dtype(dtype) or not arr.flags.c_contiguous:
        arr = np.ascontiguousarray(arr, dtype=dtype)
    return arr, arr.ctypes.data


def _prep_out(a, dtype):
    """Pointer to an output array that the library writes in place (no conversion allowed)."""
    if _is_torch(a):
        return _prep(a, dtype)[1]
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise TypeError(f"output must be a contiguous {dtype} array")
    return a.ctypes.data


def _out_like(q, shape, dtype):
    if _is_torch(q):
        import torch
        tdt = {"f4": torch.float32, "f8": torch.float64, "i4": torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=q.device)
    return np.empty(shape, dtype=dtype)


def _stream_of(a, stream):
    if stream is not None:
        return int(stream)
    if _is_torch(a) and a.is_cuda:
        import torch
        return torch.cuda.current_stream(a.device).cuda_stream
    return 0


class Dataset:
    def __init__(self, ctx: "Context", handle: int, n: int, area: float):
        self.ctx, self.handle, self.n, self.area = ctx, handle, n, area

    def destroy(self):
        if self.handle:
            _check(self.ctx.lib.aidw_destroy_dataset(self.ctx.ptr, self.handle), "destroy")
            self.handle = 0


class PreparedBatch:
    """A batch whose work list and scratch are built once and replayed as a CUDA graph."""

    def __init__(self, ctx: "Context", handle, items):
        self.ctx, self.handle, self.items = ctx, handle, items

    def launch(self, stream=None):
        st = _stream_of(self.items[0][1], stream) if self.items else 0
        _check(self.ctx.lib.aidw_batch_launch(self.ctx.ptr, self.handle, st), "batch_launch")

    def set_config(self, cfg: TuneConfig):
        _check(self.ctx.lib.aidw_batch_set_config(self.ctx.ptr, self.handle, ctypes.byref(cfg)),
               "batch_set_config")

    def config(self) -> TuneConfig:
        c = TuneConfig()
        _check(self.ctx.lib.aidw_batch_get_config(self.ctx.ptr, self.handle, ctypes.byref(c)),
               "batch_get_config")
        return c

    def autotune(self, reps: int = 2, flags: int = 0):
        """Times candidate shapes on this batch and keeps the fastest; returns (cfg, ms)."""
        c, ms = TuneConfig(), ctypes.c_double()
        _check(self.ctx.lib.aidw_batch_autotune(self.ctx.ptr, self.handle, int(reps),
                                                int(flags), ctypes.byref(c), ctypes.byref(ms)),
               "batch_autotune")
        return c, ms.value

    def destroy(self):
        if self.handle:
            _check(self.ctx.lib.aidw_batch_destroy(self.ctx.ptr, self.handle), "batch_destroy")
            self.handle = None


class Context:
    """One library context on one CUDA device (``aidw_init`` / ``aidw_shutdown``)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load()
        self._ptr = ctypes.c_void_p()
        _check(self.lib.aidw_init(ctypes.byref(self._ptr), int(device), int(hbm_budget)),
               "aidw_init")
        self.device = device
        self._keep = {}

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("context is closed")
        return self._ptr

    def close(self):
        if self._ptr:
            self.lib.aidw_shutdown(self._ptr)
            self._ptr = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- datasets --
    def create_dataset(self, x, y, z, area: float, dtype: str = "f8") -> Dataset:
        kx, px = _prep(x, dtype)
        ky, py = _prep(y, dtype)
        kz, pz = _prep(z, dtype)
        n = int(kx.shape[0])
        h = ctypes.c_int64()
        _check(self.lib.aidw_create_dataset(self.ptr, px, py, pz, n, float(area),
                                            DTYPE_F64 if dtype == "f8" else DTYPE_F32,
                                            ctypes.byref(h)), "aidw_create_dataset")
        return Dataset(self, h.value, n, area)

    # -- one-shot interpolation --
    def interpolate(self, ds: Dataset, qx, qy, params: Params | None = None, out=None,
                    out_alpha=None, out_knn=None, want_alpha=False, want_knn=False,
                    stream=None, splits=None):
        """AIDW at the queries; returns (out, out_alpha or None, out_knn or None).
        `splits` (tests) forces the plan: (phase-1 splits, phase-2 splits), 0 = planned; a
        phase-1 value of -1 forces the one-warp-per-query scan and -2 the pruned scan."""
        p = params or default_params()
        fdt = "f8" if p.precision in (F64, F64X) else "f4"
        kqx, pqx = _prep(qx, fdt)
        kqy, pqy = _prep(qy, fdt)
        m = int(kqx.shape[0])
        if out is None:
            out = _out_like(qx, (m,), fdt)
        if want_alpha and out_alpha is None:
            out_alpha = _out_like(qx, (m,), "f4")
        if want_knn and out_knn is None:
            out_knn = _out_like(qx, (m, p.k), "i4")
        ko, po = _prep(out, fdt)
        ka, pa = (None, None) if out_alpha is None else _prep(out_alpha, "f4")
        kn, pn = (None, None) if out_knn is None else _prep(out_knn, "i4")
        st = _stream_of(qx, stream)
        if splits is None:
            rc = self.lib.aidw_interpolate(self.ptr, ds.handle, pqx, pqy, m, ctypes.byref(p),
                                           po, pa, pn, st)
        else:
            rc = self.lib.aidw_debug_interpolate_splits(self.ptr, ds.handle, pqx, pqy, m,
                                                        ctypes.byref(p), po, pa, pn, st,
                                                        int(splits[0]), int(splits[1]))
        _check(rc, "aidw_interpolate")
        for keep, res in ((ko, out), (ka, out_alpha), (kn, out_knn)):
            if keep is not None and keep is not res and isinstance(res, np.ndarray):
                res[...] = keep
        return out, out_alpha, out_knn

    def interpolate_paper(self, ds: Dataset, qx, qy, params: Params | None = None,
                          version: int = VERSION_TILED, layout: int = LAYOUT_SOA, out=None,
                          out_alpha=None, want_alpha=False, stream=None):
        """AIDW by the paper's naive / tiled kernel design with SoA / AoaS data (CUDA
        tensors); returns (out, out_alpha or None)."""
        p = params or default_params()
        fdt = "f8" if p.precision in (F64, F64X) else "f4"
        kqx, pqx = _prep(qx, fdt)
        kqy, pqy = _prep(qy, fdt)
        m = int(kqx.shape[0])
        if out is None:
            out = _out_like(qx, (m,), fdt)
        if want_alpha and out_alpha is None:
            out_alpha = _out_like(qx, (m,), "f4")
        po = _prep_out(out, fdt)
        pa = None if out_alpha is None else _prep_out(out_alpha, "f4")
        _check(self.lib.aidw_interpolate_paper(self.ptr, ds.handle, pqx, pqy, m,
                                               ctypes.byref(p), po, pa, int(version),
                                               int(layout), _stream_of(qx, stream)),
               "aidw_interpolate_paper")
        return out, out_alpha

    def idw(self, ds: Dataset, qx, qy, alpha: float, precision: int = F32C, out=None,
            stream=None):
        fdt = "f8" if precision in (F64, F64X) else "f4"
        kqx, pqx = _prep(qx, fdt)
        kqy, pqy = _prep(qy, fdt)
        m = int(kqx.shape[0])
        if out is None:
            out = _out_like(qx, (m,), fdt)
        ko, po = _prep(out, fdt)
        _check(self.lib.aidw_idw(self.ptr, ds.handle, pqx, pqy, m, float(alpha), int(precision),
                                 po, _stream_of(qx, stream)), "aidw_idw")
        return out

    @staticmethod
    def _batch_items(items):
        arr = (BatchItem * max(1, len(items)))()
        for i, (ds, qx, qy, p, out, oa) in enumerate(items):
            arr[i].ds = ds.handle
            arr[i].qx = qx.data_ptr()
            arr[i].qy = qy.data_ptr()
            arr[i].m = int(qx.shape[0])
            arr[i].params = p
            arr[i].out = out.data_ptr()
            arr[i].out_alpha = oa.data_ptr() if oa is not None else None
        return arr

    def interpolate_batch(self, items, stream=None):
        """items: list of (Dataset, qx, qy, Params, out, out_alpha|None) with CUDA tensors."""
        arr = self._batch_items(items)
        st = _stream_of(items[0][1], stream) if items else 0
        _check(self.lib.aidw_interpolate_batch(self.ptr, arr, len(items), st),
               "aidw_interpolate_batch")

    def batch_create(self, items) -> "PreparedBatch":
        arr = self._batch_items(items)
        h = ctypes.c_void_p()
        _check(self.lib.aidw_batch_create(self.ptr, arr, len(items), ctypes.byref(h)),
               "aidw_batch_create")
        return PreparedBatch(self, h, items)

    # -- kernel shapes --
    def set_tune_config(self, cfg: TuneConfig):
        _check(self.lib.aidw_set_tune_config(self.ptr, ctypes.byref(cfg)), "set_tune_config")

    def tune_config(self) -> TuneConfig:
        c = TuneConfig()
        _check(self.lib.aidw_get_tune_config(self.ptr, ctypes.byref(c)), "get_tune_config")
        return c

    def autotune_interpolate(self, ds: Dataset, qx, qy, params: Params | None = None, out=None,
                             reps: int = 2, flags: int = 0):
        """Times candidate shapes on this FP32 interpolation (CUDA tensors); returns
        (cfg, ms, out)."""
        p = params or default_params()
        kqx, pqx = _prep(qx, "f4")
        kqy, pqy = _prep(qy, "f4")
        m = int(kqx.shape[0])
        if out is None:
            out = _out_like(qx, (m,), "f4")
        po = _prep_out(out, "f4")
        c, ms = TuneConfig(), ctypes.c_double()
        _check(self.lib.aidw_autotune_interpolate(self.ptr, ds.handle, pqx, pqy, m,
                                                  ctypes.byref(p), po, int(reps), int(flags),
                                                  ctypes.byref(c), ctypes.byref(ms)),
               "autotune_interpolate")
        return c, ms.value, out

    # -- serving --
    def submit(self, ds: Dataset, qx, qy, params: Params, out, out_alpha=None, out_knn=None):
        """Queue a request; returns (status, request id). The query arrays are kept alive by
        the context until the request is released; output arrays must already have the right
        dtype and be contiguous (they are written in place when the request completes)."""
        fdt = "f8" if params.precision in (F64, F64X) else "f4"
        kqx, pqx = _prep(qx, fdt)
        kqy, pqy = _prep(qy, fdt)
        po = _prep_out(out, fdt)
        pa = None if out_alpha is None else _prep_out(out_alpha, "f4")
        pn = None if out_knn is None else _prep_out(out_knn, "i4")
        rid = ctypes.c_int64()
        rc = self.lib.aidw_submit(self.ptr, ds.handle, pqx, pqy, int(len(kqx)),
                                  ctypes.byref(params), po, pa, pn, ctypes.byref(rid))
        if rc == OK:
            self._keep[rid.value] = (kqx, kqy, out, out_alpha, out_knn)
        return rc, rid.value

    def poll(self, rid: int):
        d = ctypes.c_int32()
        rc = self.lib.aidw_poll(self.ptr, int(rid), ctypes.byref(d))
        return rc, bool(d.value)

    def wait(self, rid: int, timeout_us: int = -1) -> int:
        return self.lib.aidw_wait(self.ptr, int(rid), int(timeout_us))

    def latency_us(self, rid: int) -> float:
        v = ctypes.c_double()
        _check(self.lib.aidw_request_latency_us(self.ptr, int(rid), ctypes.byref(v)), "latency")
        return v.value

    def release(self, rid: int) -> int:
        rc = self.lib.aidw_release_request(self.ptr, int(rid))
        if rc == OK:
            self._keep.pop(int(rid), None)
        return rc

    def serving_configure(self, inflight_bytes: int = 0, max_batch_requests: int = 0,
                          streams: int = 0, max_queued: int = 0):
        _check(self.lib.aidw_serving_configure(self.ptr, int(inflight_bytes),
                                               int(max_batch_requests), int(streams),
                                               int(max_queued)),
               "serving_configure")

    def serving_set_queue_limit(self, max_queued: int):
        _check(self.lib.aidw_serving_set_queue_limit(self.ptr, int(max_queued)),
               "serving_set_queue_limit")

    def serving_stats(self) -> ServingStats:
        s = ServingStats()
        _check(self.lib.aidw_serving_get_stats(self.ptr, ctypes.byref(s)), "serving_stats")
        return s

    # -- diagnostics --
    def set_profiling(self, on: bool):
        _check(self.lib.aidw_set_profiling(self.ptr, 1 if on else 0), "set_profiling")

    def kernel_times(self) -> KernelTimes:
        t = KernelTimes()
        _check(self.lib.aidw_last_kernel_times(self.ptr, ctypes.byref(t)), "kernel_times")
        return t

    def pipe_rates(self) -> PipeRates:
        r = PipeRates()
        _check(self.lib.aidw_measure_pipe_rates(self.ptr, ctypes.byref(r)), "pipe_rates")
        return r

    def check_device_errors(self) -> int:
        return self.lib.aidw_check_device_errors(self.ptr)

    def expire_wait(self, which: int, polls: int = 4096):
        """Runs a kernel whose bounded wait runs out (0: mbarrier, 1: counter)."""
        _check(self.lib.aidw_debug_expire_wait(self.ptr, int(which), int(polls)),
               "expire_wait")

    def fail_alloc_after(self, n: int):
        _check(self.lib.aidw_debug_fail_alloc_after(self.ptr, int(n)), "fail_alloc_after")
