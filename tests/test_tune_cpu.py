"""CPU checks of the kernel-shape configuration and of the autotuner's tuning cache (host-only
parts of the library: validation, the process-wide cache, and its JSON-lines file format)."""
import ctypes
import json

import pytest

from paper_1511_02186_gb300 import aidw, build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return aidw.load()


@pytest.fixture(autouse=True)
def empty_cache():
    aidw.TuneCache.clear()
    yield
    aidw.TuneCache.clear()


def test_default_shape_and_layout():
    assert ctypes.sizeof(aidw.TuneConfig) == 32
    c = aidw.tune_config()
    assert c.as_dict() == {"queries_per_thread": 2, "tile_points": 512, "knn_list": 0,
                           "split_points": 65536, "ctas_per_sm": 0,
                           "knn_queries_per_thread": 2, "unit_order": 0}
    assert aidw.tune_config_valid(c)


@pytest.mark.parametrize("field,values", [
    ("queries_per_thread", [2, 4, 8]),
    ("tile_points", [256, 512]),
    ("knn_list", [0, 16, 32]),
    ("split_points", [2048, 16384, 65536, 4194304]),
    ("ctas_per_sm", [0, 1, 3, 32]),
    ("knn_queries_per_thread", [0, 2, 4]),
    ("unit_order", [0, 1]),
])
def test_accepted_values(field, values):
    for v in values:
        assert aidw.tune_config_valid(aidw.tune_config(**{field: v})), (field, v)


@pytest.mark.parametrize("field,value", [
    ("queries_per_thread", 0), ("queries_per_thread", 3), ("queries_per_thread", 16),
    ("tile_points", 128), ("tile_points", 1024), ("tile_points", 500),
    ("knn_list", 8), ("knn_list", -1), ("knn_list", 12),
    ("split_points", 0), ("split_points", 1000), ("split_points", 2048 * 3 + 1),
    ("split_points", 8388608),
    ("ctas_per_sm", -1), ("ctas_per_sm", 33),
    ("knn_queries_per_thread", 1), ("knn_queries_per_thread", 8),
    ("unit_order", 2), ("unit_order", -1),
])
def test_rejected_values(field, value):
    assert not aidw.tune_config_valid(aidw.tune_config(**{field: value}))


def test_reserved_fields_must_be_zero():
    c = aidw.tune_config()
    c.reserved = 7
    assert not aidw.tune_config_valid(c)


def test_context_calls_reject_null_context(lib):
    c = aidw.tune_config()
    out = aidw.TuneConfig()
    ms = ctypes.c_double()
    assert lib.aidw_set_tune_config(None, ctypes.byref(c)) == aidw.ERR_INVALID_ARG
    assert lib.aidw_get_tune_config(None, ctypes.byref(out)) == aidw.ERR_INVALID_ARG
    assert lib.aidw_batch_autotune(None, None, 2, 0, ctypes.byref(out),
                                   ctypes.byref(ms)) == aidw.ERR_INVALID_ARG
    assert lib.aidw_batch_set_config(None, None, ctypes.byref(c)) == aidw.ERR_INVALID_ARG
    assert lib.aidw_autotune_interpolate(None, 1, None, None, 10, None, None, 2, 0,
                                         ctypes.byref(out), ctypes.byref(ms)) == \
        aidw.ERR_INVALID_ARG


def test_cache_put_get_clear():
    assert aidw.TuneCache.size() == 0
    assert aidw.TuneCache.get("batch dev=sm_103 x152 items=4") is None
    c = aidw.tune_config(queries_per_thread=2, split_points=32768)
    aidw.TuneCache.put("batch dev=sm_103 x152 items=4", c, 12.5)
    got = aidw.TuneCache.get("batch dev=sm_103 x152 items=4")
    assert got is not None and got[0] == c and got[1] == 12.5
    aidw.TuneCache.put("batch dev=sm_103 x152 items=4", aidw.tune_config(), 3.0)  # replaces
    assert aidw.TuneCache.size() == 1
    assert aidw.TuneCache.get("batch dev=sm_103 x152 items=4")[0] == aidw.tune_config()
    aidw.TuneCache.clear()
    assert aidw.TuneCache.size() == 0


@pytest.mark.parametrize("key", ["", 'has "quote"', "back\\slash", "tab\there", "x" * 256,
                                 "café"])
def test_cache_rejects_bad_keys(key):
    with pytest.raises(aidw.AidwError):
        aidw.TuneCache.put(key, aidw.tune_config(), 1.0)
    assert aidw.TuneCache.size() == 0


def test_cache_rejects_bad_shapes_and_times():
    with pytest.raises(aidw.AidwError):
        aidw.TuneCache.put("k", aidw.tune_config(tile_points=100), 1.0)
    with pytest.raises(aidw.AidwError):
        aidw.TuneCache.put("k", aidw.tune_config(), float("nan"))
    assert aidw.TuneCache.size() == 0


def test_save_writes_json_lines_and_load_round_trips(tmp_path):
    entries = {
        "interpolate dev=sm_103 x152 n=2^20 m=2^20 k=10": (aidw.tune_config(), 365.25),
        "batch dev=sm_103 x152 items=256 q=2^22 pairs=2^38 kmax=15":
            (aidw.tune_config(queries_per_thread=8, tile_points=256, knn_list=16,
                              split_points=131072, ctas_per_sm=3, knn_queries_per_thread=2,
                              unit_order=1),
             88.5),
    }
    for k, (c, ms) in entries.items():
        aidw.TuneCache.put(k, c, ms)
    path = tmp_path / "tune.jsonl"
    aidw.TuneCache.save(str(path))
    lines = [l for l in path.read_text().splitlines() if l.strip()]
    assert len(lines) == 2
    for l in lines:
        obj = json.loads(l)
        c, ms = entries[obj["key"]]
        assert {f: obj[f] for f in aidw.TuneConfig.FIELDS} == c.as_dict()
        assert obj["ms"] == pytest.approx(ms)
    aidw.TuneCache.clear()
    assert aidw.TuneCache.load(str(path)) == aidw.OK
    assert aidw.TuneCache.size() == 2
    for k, (c, ms) in entries.items():
        got = aidw.TuneCache.get(k)
        assert got[0] == c and got[1] == pytest.approx(ms)


def test_load_accepts_other_whitespace_and_blank_lines(tmp_path):
    path = tmp_path / "hand.jsonl"
    path.write_text(
        "\n"
        '{ "key" : "a b", "queries_per_thread":2,"tile_points" :256, "knn_list": 32 ,'
        ' "split_points": 16384, "ctas_per_sm": 1, "knn_queries_per_thread" :2,'
        ' "unit_order":1, "ms": 1e2 }\n'
        "   \n"
        + json.dumps({"key": "c", "queries_per_thread": 4, "tile_points": 512, "knn_list": 0,
                      "split_points": 65536, "ctas_per_sm": 0, "knn_queries_per_thread": 0,
                      "unit_order": 0, "ms": -1}) + "\n")
    assert aidw.TuneCache.load(str(path)) == aidw.OK
    a = aidw.TuneCache.get("a b")
    assert a[0] == aidw.tune_config(queries_per_thread=2, tile_points=256, knn_list=32,
                                    split_points=16384, ctas_per_sm=1,
                                    knn_queries_per_thread=2, unit_order=1)
    assert a[1] == 100.0
    assert aidw.TuneCache.get("c")[0] == aidw.tune_config(queries_per_thread=4,
                                                          knn_queries_per_thread=0)


@pytest.mark.parametrize("bad", [
    '{"key": "x", "queries_per_thread": 4}',                     # fields missing
    '{"key": "x", "queries_per_thread": 3, "tile_points": 512, "knn_list": 0, '
    '"split_points": 65536, "ctas_per_sm": 0, "knn_queries_per_thread": 0, "unit_order": 0, '
    '"ms": 1}',
    '{"key": "x", "queries_per_thread": 4, "tile_points": 512, "knn_list": 0, '
    '"split_points": 65536, "ctas_per_sm": 0, "knn_queries_per_thread": 0, "unit_order": 0, '
    '"ms": 1} trailing',
    '{"key": "x", "queries_per_thread": 4, "tile_points": 512, "knn_list": 0, '
    '"split_points": 65536, "ctas_per_sm": 0, "ms": 1}',         # older layout, fields missing
    "not json at all",
])
def test_load_rejects_malformed_files_without_merging(tmp_path, bad):
    good = json.dumps({"key": "good", "queries_per_thread": 4, "tile_points": 512,
                       "knn_list": 0, "split_points": 65536, "ctas_per_sm": 0,
                       "knn_queries_per_thread": 0, "unit_order": 0, "ms": 1.0})
    path = tmp_path / "bad.jsonl"
    path.write_text(good + "\n" + bad + "\n")
    assert aidw.TuneCache.load(str(path)) == aidw.ERR_INVALID_ARG
    assert aidw.TuneCache.size() == 0


def test_load_missing_file(tmp_path):
    assert aidw.TuneCache.load(str(tmp_path / "absent.jsonl")) == aidw.ERR_NOT_FOUND
