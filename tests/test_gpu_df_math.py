"""The AIDW_F64X scan's double-float pair weight against error bounds, evaluated on the GPU
through the library's probe hook: v = log2(d2 / d1sq) within 2^-46 (1 + |v|) absolute and
w = 2^(-kappa v) within 2^-44 (1 + kappa + kappa |v|) relative down to w = 2^-90 (the design
targets are about four times tighter; below, the low float of the pair turns subnormal),
exact where the coincidence rule and the nearest point rely on it (v = 0 and w = 1 at
d2 = d1sq; w = 0 far below the nearest point's weight). References: numpy's FP64 log2 / exp2 of
the FP64 ratio (errors near 2^-52), checked on a subset with 120-bit arithmetic."""
import ctypes

import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw

pytestmark = pytest.mark.gpu

DBL_MIN = np.finfo(np.float64).tiny


def probe(d2, d1sq, kappa):
    import torch
    lib = aidw.load()
    t = [torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda") for a in
         (d2, d1sq, kappa)]
    v = torch.empty_like(t[0])
    w = torch.empty_like(t[0])
    rc = lib.aidw_debug_df_weight(*(ctypes.c_void_p(a.data_ptr()) for a in t), int(t[0].numel()),
                                  ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()))
    assert rc == aidw.OK
    return v.cpu().numpy(), w.cpu().numpy()


def cases(seed, n):
    rng = np.random.default_rng(seed)
    d1sq = np.exp(rng.uniform(np.log(1e-30), np.log(1e12), n))
    ratio = np.exp(rng.uniform(0.0, np.log(1e40), n))
    ratio[: n // 8] = 1.0 + rng.uniform(0, 1e-6, n // 8)      # points next to the nearest one
    ratio[n // 8: n // 4] = 1.0 + rng.uniform(0, 1e-2, n // 8)
    d2 = d1sq * ratio
    kappa = rng.uniform(0.25, 12.0, n)
    return d2, d1sq, kappa


def test_weight_error_bounds():
    d2, d1sq, kappa = cases(11, 1 << 20)
    v, w = probe(d2, d1sq, kappa)
    v_ref = np.log2(d2 / d1sq)
    assert np.all(np.abs(v - v_ref) <= 2.0 ** -46 * (1.0 + np.abs(v_ref)))
    y = -kappa * v_ref
    w_ref = np.exp2(y)
    live = y > -90.0
    rel = np.abs(w[live] / w_ref[live] - 1.0)
    assert np.all(rel <= 2.0 ** -44 * (1.0 + kappa[live] + np.abs(y[live]))), rel.max()
    # Between 2^-90 and 2^-126 of the nearest point's weight the low float of the pair runs
    # into the float's subnormal range; the high float still carries 24 bits.
    tiny = (y <= -90.0) & (y > -125.0)
    assert np.all(np.abs(w[tiny] / w_ref[tiny] - 1.0) <= 2.0 ** -22)
    # Below 2^-127 the weight is dropped; in between it is a small positive float.
    assert np.all(w[y < -127.5] == 0.0)
    assert np.all((w >= 0.0) & (w <= 1.0 + 2.0 ** -40))


def test_against_high_precision_subset():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    d2, d1sq, kappa = cases(12, 512)
    v, w = probe(d2, d1sq, kappa)
    for a, b, k, vv, ww in zip(d2, d1sq, kappa, v, w):
        t = mp.log(mp.mpf(float(a)) / mp.mpf(float(b)), 2)
        assert abs(mp.mpf(float(vv)) - t) <= 2.0 ** -46 * (1 + abs(t))
        yy = -mp.mpf(float(k)) * t
        if yy > -90:
            assert (abs(mp.mpf(float(ww)) / mp.power(2, yy) - 1)
                    <= 2.0 ** -44 * (1 + float(k) + abs(yy)))


def test_special_values():
    # Equal distances give v = 0 and w = 1 exactly, at any scale (DBL_MIN is the coincidence
    # floor of the squared distance); the coincidence scale 2^100 leaves only those.
    d = np.array([DBL_MIN, 1.0, 3.0, 1e-300, 1e300, 0.7])
    v, w = probe(d, d, np.full(6, 2.0))
    assert np.all(v == 0.0) and np.all(w == 1.0)
    v, w = probe(np.array([DBL_MIN, DBL_MIN * (1 + 2.0 ** -52), 1e-300]), np.full(3, DBL_MIN),
                 np.full(3, 2.0 ** 100))
    assert w[0] == 1.0 and w[1] == 0.0 and w[2] == 0.0
    # Padding points (d2 = +inf) weigh nothing, whatever kappa (down to 2^-100).
    _, w = probe(np.full(3, np.inf), np.array([1.0, 1e-300, 2.0]),
                 np.array([0.025, 2.0 ** 100, 2.0 ** -100]))
    assert np.all(w == 0.0)
    # Powers of two: exact logarithms and exact weights.
    v, w = probe(np.array([8.0, 2.0 ** -40, 2.0 ** 60]), np.array([2.0, 2.0 ** -44, 1.0]),
                 np.array([1.5, 0.5, 1.0]))
    assert np.array_equal(v, [2.0, 4.0, 60.0])
    assert np.array_equal(w, [2.0 ** -3, 2.0 ** -2, 2.0 ** -60])


def test_probe_rejects_bad_arguments():
    lib = aidw.load()
    assert lib.aidw_debug_df_weight(None, None, None, -1, None, None) == aidw.ERR_INVALID_ARG
    assert lib.aidw_debug_df_weight(None, None, None, 5, None, None) == aidw.ERR_INVALID_ARG
    assert lib.aidw_debug_df_weight(None, None, None, 0, None, None) == aidw.OK
