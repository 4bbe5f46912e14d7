"""CPU checks of the C ABI: the library builds and loads, exports every function declared in
include/*.h, and fails cleanly (no crash, an error status) when no GPU is present."""
import ctypes
import glob
import os
import re

import pytest

from paper_1511_02186_gb300 import aidw, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        decl = r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(aidw_[a-z0-9_]+)\s*\("
        for m in re.finditer(decl, text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return aidw.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("aidw_init", "aidw_shutdown", "aidw_create_dataset", "aidw_destroy_dataset",
                     "aidw_interpolate", "aidw_submit", "aidw_poll", "aidw_wait",
                     "aidw_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    # The binding knows every one of them with a signature.
    assert names <= set(aidw.SIGNATURES), sorted(names - set(aidw.SIGNATURES))


def test_params_struct_layout(lib):
    assert ctypes.sizeof(aidw.Params) == 72
    p = aidw.default_params()
    assert p.k == 10 and list(p.alpha) == [1.0, 2.0, 3.0, 4.0, 5.0]
    assert p.r_min == 0.0 and p.r_max == 2.0 and p.precision == aidw.F32C


def test_status_strings(lib):
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert aidw.status_string(s) != "unknown status"
    assert aidw.status_string(12345) == "unknown status"


def test_init_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = ctypes.c_void_p()
    rc = lib.aidw_init(ctypes.byref(c), 0, 0)
    assert rc != aidw.OK and not c.value


def test_null_arguments_rejected(lib):
    assert lib.aidw_init(None, 0, 0) == aidw.ERR_INVALID_ARG
    assert lib.aidw_shutdown(None) == aidw.ERR_INVALID_ARG
    assert lib.aidw_interpolate(None, 1, None, None, 0, None, None, None, None, None) == \
        aidw.ERR_INVALID_ARG
    d = ctypes.c_int32()
    assert lib.aidw_poll(None, 1, ctypes.byref(d)) == aidw.ERR_INVALID_ARG


def test_binding_refuses_missing_library(tmp_path):
    with pytest.raises(ImportError):
        aidw.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(aidw.load, "__wrapped__") \
            else _fresh_load(str(tmp_path / "nope.so"))


def _fresh_load(path):
    saved = aidw._lib
    aidw._lib = None
    try:
        return aidw.load(path)
    finally:
        aidw._lib = saved
