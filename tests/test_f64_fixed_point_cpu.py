"""The FP64 path's fixed-point log2 / exp2, as a bit-exact model of the integer steps
(tests/f64_fixed_model.py), against 120-bit references on the CPU: random arguments over the
whole range, both ends of every table interval, the rounding points of exp2's reduction, and the
exact values the coincidence rule and powers of two rely on. A GPU test checks that the library
gives the model's doubles bit for bit, so these bounds hold for the kernels."""
import math
import random

import pytest

import f64_fixed_model as fm

mp = pytest.importorskip("mpmath")
DBL_MIN = 2.2250738585072014e-308
ULP1 = 2.0 ** -52


@pytest.fixture(scope="module")
def tabs():
    return fm.load_tables()


@pytest.fixture(scope="module")
def prec():
    old = mp.mp.prec
    mp.mp.prec = 120
    yield
    mp.mp.prec = old


def log2_args(seed=1, n=3000):
    rnd = random.Random(seed)
    xs = [math.exp(rnd.uniform(math.log(DBL_MIN), math.log(1e300))) for _ in range(n)]
    xs += [1 + rnd.uniform(-1e-3, 1e-3) for _ in range(n // 3)]
    for j in range(0, 1024, 3):  # both ends of table intervals, at several exponents
        for e in (-1000, -3, 0, 7, 512):
            xs.append((1 + j / 1024) * 2.0 ** e)
            xs.append(math.nextafter((1 + (j + 1) / 1024) * 2.0 ** e, 0))
    return xs


def exp2_args(seed=2, n=3000):
    rnd = random.Random(seed)
    ys = [rnd.uniform(-1020.9, 8.0) for _ in range(n)]
    ys += [rnd.uniform(-1e-3, 1e-3) for _ in range(n // 3)]
    for k in [rnd.randint(-1020 * 1024, 8 * 1024) for _ in range(300)] + list(range(-600, 600)):
        for y in (k / 1024, (k + 0.5) / 1024, (k - 0.5) / 1024):
            ys += [y, math.nextafter(y, math.inf), math.nextafter(y, -math.inf)]
    ys += [2.0 ** rnd.uniform(-60, -11) * rnd.choice([-1, 1]) for _ in range(500)]
    return [y for y in ys if -1020.99 < y < 8.0]


def test_log2_within_one_ulp_of_max_1_and_log2(tabs, prec):
    """Absolute error at most 0.75 ulp of max(1, |log2 x|): the fraction's rounding to 2^-53 and
    the final rounding to a double (the polynomials' own error is below 2^-58)."""
    worst = 0.0
    for x in log2_args():
        t = mp.log(mp.mpf(x), 2)
        v = fm.log2_fx(x, tabs)
        worst = max(worst, float(abs(mp.mpf(v) - t) / max(1, abs(t))) / ULP1)
    assert worst <= 0.75, worst


def test_exp2_within_an_ulp_and_a_quarter(tabs, prec):
    """Relative error at most 1.25 ulps (the quadratic's error, about 0.6 ulp at most, and the
    final rounding); the 96-bit fixed-point weight within the same bound plus 2^-95."""
    worst = 0.0
    for y in exp2_args():
        t = mp.power(2, mp.mpf(y))
        w, w96 = fm.exp2_fx(y, tabs)
        worst = max(worst, float(abs(mp.mpf(w) / t - 1)) / ULP1)
        if y <= 0.5:
            assert abs(mp.mpf(w96) / mp.mpf(2) ** 96 - t) <= mp.mpf(2) ** -95 + 1.25 * ULP1 * t, y
    assert worst <= 1.25, worst


def test_exact_values(tabs):
    """log2 of powers of two and of the smallest normal double (the coincidence rule's d^2) are
    exact; exp2 of 0 is 1 (the nearest point's weight), of integers a power of two, of -1021 and
    below 0; log2 of +inf is +inf."""
    for e in (-1022, -1000, -1, 0, 1, 7, 1000):
        assert fm.log2_fx(2.0 ** e, tabs) == float(e)
    assert fm.log2_fx(math.inf, tabs) == math.inf
    assert fm.exp2_fx(0.0, tabs) == (1.0, 1 << 96)
    for e in (-1020, -50, -1, 1, 7):
        assert fm.exp2_fx(float(e), tabs)[0] == 2.0 ** e
    assert fm.exp2_fx(-1021.0, tabs)[0] == 0.0 and fm.exp2_fx(-1e300, tabs)[0] == 0.0
    assert fm.exp2_fx(-math.inf, tabs)[0] == 0.0


def _truncating_fx52_to_double(a):
    """fx52_to_double without its rounding bit (the significand truncated)."""
    s = (a & fm.M64) & (1 << 63)
    m = (-a if a < 0 else a) & fm.M64
    lz = fm.clz64(m | 1)
    sig = ((m << lz) & fm.M64) >> 11
    b = (((1034 - lz) << 52) + sig - (1 << 52)) & fm.M64
    return 0.0 if m == 0 else fm.from_bits(b | s)


MISTAKES = {
    # a product's high word shifted one bit too little (a wrong fixed-point scale)
    "product_scale": ("fx_mul", lambda p, v: ((p * v) >> 64) >> 8),
    # the innermost Horner term of log2 and exp2 dropped
    "inner_term_dropped": ("fx_mul32", lambda p, v: 0),
    # log2's result truncated instead of rounded to a double
    "log2_truncated": ("fx52_to_double", _truncating_fx52_to_double),
}


@pytest.mark.parametrize("mistake", sorted(MISTAKES))
def test_planted_mistakes_are_caught(tabs, prec, mistake, monkeypatch):
    """Each planted mistake in the model breaks one of the bounds above."""
    name, fn = MISTAKES[mistake]
    monkeypatch.setattr(fm, name, fn)
    caught = False
    for x in log2_args(n=600):
        t = mp.log(mp.mpf(x), 2)
        if abs(mp.mpf(fm.log2_fx(x, tabs)) - t) > 0.75 * ULP1 * max(1, abs(t)):
            caught = True
            break
    if not caught:
        for y in exp2_args(n=600):
            t = mp.power(2, mp.mpf(y))
            w, _ = fm.exp2_fx(y, tabs)
            if abs(mp.mpf(w) / t - 1) > 1.25 * ULP1:
                caught = True
                break
    assert caught, mistake
