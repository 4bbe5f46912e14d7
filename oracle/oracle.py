"""ctypes front end of the plain-C FP64 AIDW oracle (``aidw_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU-baseline leg of the
benchmark. Every function states the passage of Mei, Xu & Xu (arXiv 1511.02186) it follows;
the arithmetic itself is in ``aidw_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aidw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: every product and sum is rounded separately, as the oracle requires.
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           "-std=c11", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle to ``oracle/_build/liboracle.so`` if missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    p = ctypes.c_void_p
    lib.aidw_oracle_r_exp.restype = d
    lib.aidw_oracle_r_exp.argtypes = [i64, d]
    lib.aidw_oracle_mu.restype = d
    lib.aidw_oracle_mu.argtypes = [d, d, d]
    lib.aidw_oracle_alpha.restype = d
    lib.aidw_oracle_alpha.argtypes = [d, p]
    lib.aidw_oracle_interpolate.restype = i32
    lib.aidw_oracle_interpolate.argtypes = [p, p, p, i64, d, p, p, i64, i32, p, d, d,
                                            p, p, p, p, p, i32]
    lib.aidw_oracle_idw.restype = i32
    lib.aidw_oracle_idw.argtypes = [p, p, p, i64, p, p, i64, d, p, p, i32]
    lib.aidw_oracle_knn.restype = i32
    lib.aidw_oracle_knn.argtypes = [p, p, i64, p, p, i64, i32, p, p]
    return lib


def load_library(path: str):
    """Load an oracle build from ``path`` (the tests also load deliberately broken copies)."""
    return _bind(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def r_exp(n: int, area: float, lib=None) -> float:
    """Eq. 2: expected nearest-neighbour distance for n points on area A."""
    return (lib or _load()).aidw_oracle_r_exp(int(n), float(area))


def mu_of_R(R: float, r_min: float = 0.0, r_max: float = 2.0, lib=None) -> float:
    """Eq. 5: fuzzy membership of the NN statistic (defaults R_min = 0, R_max = 2, Sec. 2.2)."""
    return (lib or _load()).aidw_oracle_mu(float(R), float(r_min), float(r_max))


def alpha_of_mu(mu: float, levels, lib=None) -> float:
    """Eq. 6: triangular mapping of mu_R onto the five alpha levels."""
    lv = _f64(levels)
    assert lv.shape == (5,)
    return (lib or _load()).aidw_oracle_alpha(float(mu), _ptr(lv))


def knn(x, y, qx, qy, k: int, lib=None):
    """Sec. 3.1.2: k nearest data points per query. Returns (idx[m,k] int64, d2[m,k] f64),
    ascending by (d2, index)."""
    x, y, qx, qy = _f64(x), _f64(y), _f64(qx), _f64(qy)
    m = qx.shape[0]
    idx = np.empty((m, k), dtype=np.int64)
    d2 = np.empty((m, k), dtype=np.float64)
    rc = (lib or _load()).aidw_oracle_knn(_ptr(x), _ptr(y), x.shape[0], _ptr(qx), _ptr(qy), m, k,
                                 _ptr(idx), _ptr(d2))
    if rc != 0:
        raise ValueError(f"oracle knn rejected its arguments (code {rc})")
    return idx, d2


def interpolate(x, y, z, area: float, qx, qy, k: int, levels=(1.0, 2.0, 3.0, 4.0, 5.0),
                r_min: float = 0.0, r_max: float = 2.0, threads: int | None = None,
                lib=None) -> dict:
    """AIDW (Sec. 2.2 phase 1: kNN, Eq. 2-6; phase 2: Eq. 1 over all n points).

    Returns a dict of float64/int64 arrays: ``z`` (prediction), ``alpha``, ``R`` (NN
    statistic), ``knn`` [m,k], and ``scale`` = sum(w|z|)/sum(w), the condition scale used as
    the relative-error denominator together with |z|.
    """
    x, y, z, qx, qy = _f64(x), _f64(y), _f64(z), _f64(qx), _f64(qy)
    lv = _f64(levels)
    n, m = x.shape[0], qx.shape[0]
    out = {
        "z": np.empty(m), "alpha": np.empty(m), "R": np.empty(m),
        "knn": np.empty((m, k), dtype=np.int64), "scale": np.empty(m),
    }
    rc = (lib or _load()).aidw_oracle_interpolate(
        _ptr(x), _ptr(y), _ptr(z), n, float(area), _ptr(qx), _ptr(qy), m, int(k), _ptr(lv),
        float(r_min), float(r_max), _ptr(out["z"]), _ptr(out["alpha"]), _ptr(out["R"]),
        _ptr(out["knn"]), _ptr(out["scale"]), int(threads or default_threads()))
    if rc != 0:
        raise ValueError(f"oracle interpolate rejected its arguments (code {rc})")
    return out


def idw(x, y, z, qx, qy, alpha: float, threads: int | None = None, lib=None) -> dict:
    """Standard IDW, Eq. 1 with a constant alpha, over all n points (Sec. 2.1)."""
    x, y, z, qx, qy = _f64(x), _f64(y), _f64(z), _f64(qx), _f64(qy)
    m = qx.shape[0]
    out = {"z": np.empty(m), "scale": np.empty(m)}
    rc = (lib or _load()).aidw_oracle_idw(_ptr(x), _ptr(y), _ptr(z), x.shape[0], _ptr(qx), _ptr(qy), m,
                                 float(alpha), _ptr(out["z"]), _ptr(out["scale"]),
                                 int(threads or default_threads()))
    if rc != 0:
        raise ValueError(f"oracle idw rejected its arguments (code {rc})")
    return out
