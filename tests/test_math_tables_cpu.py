"""The constant tables of the phase-2 log2 / exp2, checked on the CPU against their definitions
with 120-bit arithmetic: csrc/f64_math_tables.inc (the FP64 scan: every entry the nearest double
to its value) and csrc/df_math_tables.inc (the FP64X scan: every pair hi + lo within 2^-48 of
its value, relative, with hi the nearest float and |lo| at most half an ulp of hi). The files
are also what the generator script writes, bit for bit."""
import importlib.util
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1511_02186_gb300", "csrc")


def parse(path):
    """name -> list of values (arrays) or value (scalars) of a table file."""
    text = open(path).read()
    out = {}
    for m in re.finditer(r"__device__ (?:__constant__|const) (?:double|float) (\w+)\[(\d+)\] = "
                         r"\{(.*?)\};", text, re.S):
        vals = [float.fromhex(t.strip().rstrip("f")) for t in m.group(3).split(",") if t.strip()]
        assert len(vals) == int(m.group(2)), m.group(1)
        out[m.group(1)] = vals
    for m in re.finditer(r"constexpr (?:double|float) (\w+) = ([^;]+);", text):
        out[m.group(1)] = float.fromhex(m.group(2).strip().rstrip("f"))
    return out


def ulp64(x):
    return float(np.spacing(np.float64(abs(x)))) if x != 0 else 2.0 ** -1074


def ulp32(x):
    return float(np.spacing(np.float32(abs(x)))) if x != 0 else 2.0 ** -149


def nearest_double(v, exact):
    return abs(mp.mpf(v) - exact) <= mp.mpf(ulp64(v)) / 2


def good_pair(h, l, exact):
    """hi the nearest float (to within the double rounding the generator goes through), lo at
    most half an ulp of hi, and the pair within 2^-48 of the value, relative."""
    return (abs(mp.mpf(h) - exact) <= mp.mpf(ulp32(h)) * (0.5 + 2.0 ** -28) and
            abs(l) <= ulp32(h) / 2 and
            abs(mp.mpf(h) + mp.mpf(l) - exact) <= abs(exact) * mp.mpf(2) ** -48)


@pytest.fixture(scope="module")
def prec():
    old = mp.mp.prec
    mp.mp.prec = 120
    yield
    mp.mp.prec = old


def test_fp64_tables_are_nearest_doubles(prec):
    t = parse(os.path.join(CSRC, "f64_math_tables.inc"))
    ln2 = mp.log(2)
    assert len(t["kLog2F"]) == 2048 and len(t["kInvF"]) == 2048 and len(t["kExp2J"]) == 2048
    for j in range(2048):
        f = 1 + mp.mpf(j) / 2048
        assert nearest_double(t["kLog2F"][j], mp.log(f) / ln2), j
        assert nearest_double(t["kInvF"][j], 1 / f), j
        T = mp.power(2, mp.mpf(j) / 2048)
        assert nearest_double(t["kExp2J"][j], T), j
        # e^(r ln 2) = sum (r ln 2)^i / i!, multiplied out with T_j
        for i in range(1, 4):
            assert nearest_double(t[f"kExp2C{i}"][j], T * ln2 ** i / mp.factorial(i)), (i, j)
    # log2(1 + r) = sum (-1)^(i+1) r^i / (i ln 2)
    for i in range(1, 5):
        assert nearest_double(t[f"kL2C{i}"], mp.mpf((-1) ** (i + 1)) / (i * ln2)), i
    assert "kL2C5" not in t
    # The exact anchors the coincidence rule and powers of two rely on.
    assert t["kLog2F"][0] == 0.0 and t["kInvF"][0] == 1.0 and t["kExp2J"][0] == 1.0
    assert t["kInvF"][1024] == float.fromhex("0x1.5555555555555p-1")  # 1 / 1.5, rounded


def test_double_float_tables_are_accurate_pairs(prec):
    t = parse(os.path.join(CSRC, "df_math_tables.inc"))
    ln2 = mp.log(2)
    g, l2f, e2 = t["kDfInvFLn2"], t["kDfLog2F"], t["kDfExp2K"]
    assert len(g) == 512 and len(l2f) == 512 and len(e2) == 256
    for j in range(256):
        f = 1 + mp.mpf(j) / 256
        assert good_pair(g[2 * j], g[2 * j + 1], 1 / (f * ln2)), j
        assert good_pair(l2f[2 * j], l2f[2 * j + 1], mp.log(f) / ln2) or j == 0, j
    assert l2f[0] == 0.0 and l2f[1] == 0.0
    for k in range(128):
        assert good_pair(e2[2 * k], e2[2 * k + 1], mp.power(2, mp.mpf(k) / 128)), k
    assert e2[0] == 1.0 and e2[1] == 0.0
    assert good_pair(t["kDfC2h"], t["kDfC2l"], -ln2 / 2)
    assert good_pair(t["kDfLn2h"], t["kDfLn2l"], ln2)
    for i in range(3, 7):
        c = mp.mpf((-1) ** (i + 1)) * ln2 ** (i - 1) / i
        v = t[f"kDfC{i}"]
        assert abs(mp.mpf(v) - c) <= mp.mpf(ulp32(v)) * 0.5 * (1 + 2.0 ** -28), i


def test_generator_reproduces_the_committed_files(tmp_path, prec):
    spec = importlib.util.spec_from_file_location(
        "gen_tables", os.path.join(CSRC, "gen_f64_math_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    gen.HERE = str(tmp_path)
    gen.main()
    for name in ("f64_math_tables.inc", "df_math_tables.inc"):
        assert (tmp_path / name).read_text() == open(os.path.join(CSRC, name)).read(), name
