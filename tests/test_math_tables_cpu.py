"""The constant tables of the phase-2 log2 / exp2, checked on the CPU against their definitions
with 120-bit arithmetic: csrc/f64_math_tables.inc (the FP64 scan, in fixed point: every entry
the nearest integer to its value * 2^62) and csrc/df_math_tables.inc (the FP64X scan: every pair
hi + lo within 2^-48 of its value, relative, with hi the nearest float and |lo| at most half an
ulp of hi). The files are also what the generator script writes, bit for bit."""
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
    for m in re.finditer(r"__device__ const long long (\w+)\[(\d+)\] = \{(.*?)\};", text, re.S):
        vals = [int(t.strip().rstrip("L"), 16) for t in m.group(3).split(",") if t.strip()]
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


def test_fp64_tables_are_accurate(prec):
    """Fixed point at 2^62, every entry positive (log2's coefficients as magnitudes of alternating
    signs): log2 F_j and T_j are the nearest integers to their values * 2^62;
    each entry's polynomial, with its coefficients as stored, is within its stated bound of the
    function at 9 points of its interval (evaluated exactly in 120-bit arithmetic):
    |log2 F_j + u q_j(u) - log2(F_j + u)| below 2^-58 for u in [0, 2^-10] (the cubic's error,
    about 2^-58.5, and the coefficients' rounding), |T_j + r q_j(r) - T_j 2^r| below 2^-52.5 T_j
    for r in [-2^-11, 2^-11] (the quadratic's error, at most 2^-52.7)."""
    t = parse(os.path.join(CSRC, "f64_math_tables.inc"))
    ln2 = mp.log(2)
    one = mp.mpf(2) ** 62
    for name in ("kFxLog2F", "kFxL2A1", "kFxL2A2", "kFxL2A3", "kFxL2A4", "kFxExp2T", "kFxExp2E1",
                 "kFxExp2E2", "kFxExp2E3"):
        assert len(t[name]) == 1024, name
        assert all(0 <= v < 2 ** 63 for v in t[name]), name
    h, he = mp.mpf(2) ** -10, mp.mpf(2) ** -11
    us = [h * i / 8 for i in range(9)]
    rs = [he * (i - 4) / 4 for i in range(9)]
    for j in range(1024):
        F = 1 + mp.mpf(j) / 1024
        assert abs(t["kFxLog2F"][j] - mp.log(F) / ln2 * one) <= 0.5, j
        a = [mp.mpf(t[f"kFxL2A{i}"][j]) / one for i in range(1, 5)]
        for u in us:
            p = mp.mpf(t["kFxLog2F"][j]) / one + u * (a[0] - u * (a[1] - u * (a[2] - u * a[3])))
            assert abs(p - mp.log(F + u) / ln2) < mp.mpf(2) ** -58, (j, u)
        T = mp.power(2, mp.mpf(j) / 1024)
        assert abs(t["kFxExp2T"][j] - T * one) <= 0.5, j
        e = [mp.mpf(t[f"kFxExp2E{i}"][j]) / one for i in range(1, 4)]
        for r in rs:
            p = mp.mpf(t["kFxExp2T"][j]) / one + r * (e[0] + r * (e[1] + r * e[2]))
            assert abs(p - T * mp.power(2, r)) < T * mp.mpf(2) ** -52.5, (j, r)
    # The exact anchors the coincidence rule and powers of two rely on.
    assert t["kFxLog2F"][0] == 0 and t["kFxExp2T"][0] == 2 ** 62


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
