"""The FP64 path's table-driven log2 / exp2 against error bounds, evaluated on the GPU through
the library's probe hook: log2 within 2 ulps of max(1, |log2 x|) in absolute terms (the
accuracy the weights of Eq. 1 need: log2 is scaled by alpha/2 and exponentiated), exp2 within
4 ulps relative, exact at the points the coincidence rule relies on (log2 of the smallest
normal double, exp2(0)), and the limits the scan relies on (log2(+inf) = +inf, exp2 of very
negative arguments = 0). References: numpy's log2 / exp2 (within an ulp), checked on a subset
with 120-bit arithmetic."""
import ctypes

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw

pytestmark = pytest.mark.gpu

DBL_MIN = np.finfo(np.float64).tiny
ULP1 = 2.0 ** -52


def probe(x, y):
    import torch
    lib = aidw.load()
    tx = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    ty = torch.as_tensor(y, dtype=torch.float64, device="cuda")
    lx = torch.empty_like(tx)
    ey = torch.empty_like(ty)
    rc = lib.aidw_debug_f64_log2_exp2(ctypes.c_void_p(tx.data_ptr()),
                                      ctypes.c_void_p(ty.data_ptr()), int(tx.numel()),
                                      ctypes.c_void_p(lx.data_ptr()),
                                      ctypes.c_void_p(ey.data_ptr()))
    assert rc == aidw.OK
    return lx.cpu().numpy(), ey.cpu().numpy()


def test_log2_exp2_error_bounds():
    rng = np.random.default_rng(3)
    n = 1 << 20
    x = np.exp(rng.uniform(np.log(DBL_MIN), np.log(1e300), n))
    x[:4096] = 1.0 + rng.uniform(-1e-3, 1e-3, 4096)          # near 1: log2 near 0
    x[4096:8192] = 2.0 ** rng.integers(-1022, 1000, 4096)     # powers of two: exact results
    y = rng.uniform(-1020.9, 8.0, n)
    y[:4096] = rng.uniform(-1e-3, 1e-3, 4096)
    lx, ey = probe(x, y)
    ref_l = np.log2(x)
    err_l = np.abs(lx - ref_l) / np.maximum(1.0, np.abs(ref_l))
    assert err_l.max() <= 2 * ULP1, err_l.max()
    assert np.array_equal(lx[4096:8192], ref_l[4096:8192])   # exact on powers of two
    ref_e = np.exp2(y)
    err_e = np.abs(ey / ref_e - 1.0)
    assert err_e.max() <= 4 * ULP1 / 2, err_e.max()


def test_against_high_precision_subset():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(4)
    x = np.exp(rng.uniform(np.log(DBL_MIN), np.log(1e300), 512))
    y = rng.uniform(-1020.9, 4.0, 512)
    lx, ey = probe(x, y)
    for a, v in zip(x, lx):
        t = mp.log(mp.mpf(float(a)), 2)
        assert abs(mp.mpf(float(v)) - t) <= 2 * ULP1 * max(1, abs(t))
    for b, v in zip(y, ey):
        t = mp.power(2, mp.mpf(float(b)))
        assert abs(mp.mpf(float(v)) / t - 1) <= 2 * ULP1


def test_special_values():
    x = np.array([DBL_MIN, 1.0, 2.0, 0.5, np.inf, 1e308, 3.0])
    y = np.array([0.0, -1.0, 1.0, -1021.0, -1e300, -np.inf, -1020.5])
    lx, ey = probe(x, y)
    assert lx[0] == -1022.0 and lx[1] == 0.0 and lx[2] == 1.0 and lx[3] == -1.0
    assert np.isposinf(lx[4])
    assert abs(lx[5] - np.log2(1e308)) <= 2 * ULP1 * np.log2(1e308)
    assert ey[0] == 1.0 and ey[1] == 0.5 and ey[2] == 2.0
    assert ey[3] == 0.0 and ey[4] == 0.0 and ey[5] == 0.0
    assert ey[6] > 0.0 and abs(ey[6] / np.exp2(-1020.5) - 1) <= 2 * ULP1


def test_integer_reduction_edges():
    """The steps done on the integer pipe at their edges. exp2: arguments at and around the
    rounding points of k = round(1024 y) (k/1024 +- half a step, +- an ulp), arguments so small
    that k = 0 (|1024 y| < 1/4), negative and positive; log2: mantissas whose bits below the
    10-bit table index are all ones or a single one, and the neighbours of powers of two. All
    within the same bounds as above."""
    rng = np.random.default_rng(5)
    k = rng.integers(-1020 * 1024, 8 * 1024, 4096).astype(np.float64)
    step = 1.0 / 1024
    y = np.concatenate([k * step, (k + 0.5) * step, (k - 0.5) * step,
                        np.nextafter((k + 0.5) * step, np.inf),
                        np.nextafter((k + 0.5) * step, -np.inf),
                        rng.uniform(-2.0 ** -13, 2.0 ** -13, 2048),
                        2.0 ** rng.uniform(-60, -11, 2048) * rng.choice([-1.0, 1.0], 2048)])
    y = y[(y > -1020.99) & (y < 8.0)]
    e = rng.integers(-1000, 1000, 2048).astype(np.float64)
    p2 = 2.0 ** e
    mant = rng.integers(0, 1024, 2048)
    ones = (1.0 + mant / 1024.0 + (2.0 ** -10 - 2.0 ** -52)) * p2   # low 42 bits all ones
    one = (1.0 + mant / 1024.0 + 2.0 ** -52) * p2                   # a single low bit
    x = np.concatenate([ones, one, np.nextafter(p2, np.inf), np.nextafter(p2, 0.0)])
    n = max(len(x), len(y))
    xs = np.resize(x, n)
    ys = np.resize(y, n)
    lx, ey = probe(xs, ys)
    ref_l = np.log2(xs)
    err_l = np.abs(lx - ref_l) / np.maximum(1.0, np.abs(ref_l))
    assert err_l.max() <= 2 * ULP1, err_l.max()
    ref_e = np.exp2(ys)
    err_e = np.abs(ey / ref_e - 1.0)
    assert err_e.max() <= 4 * ULP1 / 2, err_e.max()
    # k/1024 itself: exact up to the table entry's rounding (r = 0).
    lk, ek = probe(np.ones(16), np.arange(-8, 8) * step)
    assert np.all(np.abs(ek / np.exp2(np.arange(-8, 8) * step) - 1.0) <= ULP1)


def test_kernels_match_the_integer_model_bit_for_bit():
    """For every argument the library's log2 / exp2 give the doubles of the bit-exact model of
    their integer steps (tests/f64_fixed_model.py), whose accuracy the CPU tests pin against
    120-bit references: random arguments over the whole range, both ends of table intervals,
    the rounding points of exp2's reduction, tiny and exactly representable arguments."""
    import f64_fixed_model as fm
    t = fm.load_tables()
    rng = np.random.default_rng(6)
    x = np.exp(rng.uniform(np.log(DBL_MIN), np.log(1e300), 12000))
    j = rng.integers(0, 1024, 4000)
    e = 2.0 ** rng.integers(-1022, 1000, 4000)
    x = np.concatenate([x, (1.0 + j / 1024.0) * e,
                        np.nextafter((1.0 + (j + 1) / 1024.0) * e, 0.0), [DBL_MIN, 1.0, np.inf]])
    k = rng.integers(-1020 * 1024, 8 * 1024, 4000).astype(np.float64) / 1024.0
    y = np.concatenate([rng.uniform(-1020.9, 8.0, 12000), k, k + 0.5 / 1024,
                        np.nextafter(k + 0.5 / 1024, -np.inf),
                        2.0 ** rng.uniform(-60, -11, 3000) * rng.choice([-1.0, 1.0], 3000),
                        [0.0, -1.0, -1021.0, -1e300]])
    y = y[y < 8.0]
    n = max(len(x), len(y))
    xs, ys = np.resize(x, n), np.resize(y, n)
    lx, ey = probe(xs, ys)
    ml = np.array([fm.log2_fx(float(a), t) for a in xs])
    me = np.array([fm.exp2_fx(float(b), t)[0] for b in ys])
    bad_l = np.flatnonzero(ml.view(np.int64) != lx.view(np.int64))
    bad_e = np.flatnonzero(me.view(np.int64) != ey.view(np.int64))
    assert bad_l.size == 0, [(xs[i], lx[i], ml[i]) for i in bad_l[:5]]
    assert bad_e.size == 0, [(ys[i], ey[i], me[i]) for i in bad_e[:5]]
