"""Pins for the FP64 CPU oracle: it is checked against things other than itself.

* hand-derived closed forms of Eq. 2, Eq. 5 and Eq. 6 (tests/golden/membership_hand_values.json)
* hand-built worked examples whose R lands on exact closed forms (tests/golden/worked_examples.json)
* kNN (Sec. 3.1.2) against a brute-force full sort and against the printed procedure run step by
  step in Python, on tie-heavy lattice inputs
* the Clark-Evans statistic: for a uniform random pattern the mean k-NN statistic R of Eq. 4 has a
  closed form from the Poisson nearest-neighbour distribution
* invariants of the weighted mean of Eq. 1 (bounds, constants, permutations, scaling) and its
  textbook special case (all levels equal: Shepard IDW)
* a meta-test that plants plausible mistakes in a copy of the oracle and checks that the pins
  catch every one of them
"""
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1511_02186_gb300 import workloads

NS = {"sqrt": math.sqrt, "sin": math.sin, "cos": math.cos, "pi": math.pi}
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def closed(expr: str) -> float:
    return float(eval(expr, {"__builtins__": {}}, NS))


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------------------------
# Independent references written in the tests (no oracle code)
# ---------------------------------------------------------------------------------------------

def brute_knn(x, y, qx, qy, k):
    """k smallest (d2, index) per query by a full lexicographic sort."""
    out = []
    for a, b in zip(qx, qy):
        d2 = (a - x) * (a - x) + (b - y) * (b - y)
        order = np.lexsort((np.arange(len(x)), d2))
        out.append(order[:k])
    return np.array(out)


def printed_knn_procedure(x, y, qx, qy, k):
    """Sec. 3.1.2 run literally: Step 1 the first k distances, Step 2 sort them ascending,
    Step 3 for every further point, replace the k-th if strictly closer and swap neighbours
    from the k-th toward the first until sorted again."""
    res = []
    for a, b in zip(qx, qy):
        dist = lambda i: (a - x[i]) * (a - x[i]) + (b - y[i]) * (b - y[i])  # noqa: E731
        lst = sorted(((dist(i), i) for i in range(k)), key=lambda t: (t[0], t[1]))
        for i in range(k, len(x)):
            d = dist(i)
            if d < lst[k - 1][0]:
                lst[k - 1] = (d, i)
                j = k - 1
                while j > 0 and lst[j][0] < lst[j - 1][0]:
                    lst[j], lst[j - 1] = lst[j - 1], lst[j]
                    j -= 1
        res.append([i for _, i in lst])
    return np.array(res)


def clark_evans_mean_R(k: int) -> float:
    """E[R] for a Poisson pattern: E[D_j] = Gamma(j + 1/2) / (Gamma(j) sqrt(pi lambda)) and
    r_exp = 1 / (2 sqrt(lambda)), so E[R] = (2/sqrt(pi)) (1/k) sum_j Gamma(j+1/2)/Gamma(j)."""
    s = sum(math.exp(math.lgamma(j + 0.5) - math.lgamma(j)) for j in range(1, k + 1))
    return 2.0 / math.sqrt(math.pi) * s / k


def lattice_case(seed, n_side=10, m=40):
    rng = np.random.default_rng(seed)
    gx, gy = np.meshgrid(np.arange(n_side, dtype=float), np.arange(n_side, dtype=float))
    perm = rng.permutation(n_side * n_side)
    x, y = gx.ravel()[perm], gy.ravel()[perm]
    qx = rng.integers(0, 2 * n_side, m) / 2.0
    qy = rng.integers(0, 2 * n_side, m) / 2.0
    return x, y, qx, qy


# ---------------------------------------------------------------------------------------------
# Pin suite, runnable against any build of the oracle (the real one or a planted mistake)
# ---------------------------------------------------------------------------------------------

def pin_failures(lib=None, quick=False):
    """Run every pin against ``lib`` and return a list of failure messages."""
    fails = []
    g = load_golden("membership_hand_values.json")
    for c in g["eq2_r_exp"]:
        v = oracle.r_exp(c["n"], c["area"], lib=lib)
        if not math.isclose(v, closed(c["closed_form"]), rel_tol=1e-15):
            fails.append(f"Eq.2 n={c['n']} A={c['area']}: {v}")
    for c in g["eq5_mu"]:
        v = oracle.mu_of_R(c["R"], c["r_min"], c["r_max"], lib=lib)
        if not math.isclose(v, closed(c["closed_form"]), rel_tol=1e-14, abs_tol=1e-15):
            fails.append(f"Eq.5 R={c['R']} rmin={c['r_min']}: {v}")
    lv = g["eq6_alpha"]["levels"]
    for c in g["eq6_alpha"]["cases"]:
        v = oracle.alpha_of_mu(c["mu"], lv, lib=lib)
        if not math.isclose(v, closed(c["closed_form"]), rel_tol=1e-14):
            fails.append(f"Eq.6 mu={c['mu']}: {v}")

    w = load_golden("worked_examples.json")
    for c in w["cases"]:
        r = oracle.interpolate(c["x"], c["y"], c["z"], c["area"], c["qx"], c["qy"], c["k"],
                               c["levels"], threads=1, lib=lib)
        if not math.isclose(r["R"][0], closed(c["R"]), rel_tol=1e-14, abs_tol=1e-15):
            fails.append(f"{c['name']}: R {r['R'][0]}")
        if not math.isclose(r["alpha"][0], closed(c["alpha"]), rel_tol=1e-14):
            fails.append(f"{c['name']}: alpha {r['alpha'][0]}")
        if not math.isclose(r["z"][0], closed(c["z_out"]), rel_tol=1e-14):
            fails.append(f"{c['name']}: Z {r['z'][0]}")
        if r["knn"].tolist() != c["knn"]:
            fails.append(f"{c['name']}: knn {r['knn'].tolist()}")
        if not math.isclose(r["scale"][0], closed(c["scale"]), rel_tol=1e-14):
            fails.append(f"{c['name']}: S* {r['scale'][0]}")

    # S* = sum(w|z|)/sum(w) is the weighted mean of |z| under the same weights: it equals Z
    # for z >= 0, equals the Z of |z| for any z, and ignores the sign of z.
    wl = workloads.small_case(17, 300, 40, pattern="clustered")
    zs = wl.z - np.median(wl.z)  # both signs
    for zz in (np.abs(zs) + 0.5, zs):
        r = oracle.interpolate(wl.x, wl.y, zz, wl.area, wl.qx, wl.qy, wl.k, threads=1, lib=lib)
        ra = oracle.interpolate(wl.x, wl.y, np.abs(zz), wl.area, wl.qx, wl.qy, wl.k, threads=1,
                                lib=lib)
        rn = oracle.interpolate(wl.x, wl.y, -zz, wl.area, wl.qx, wl.qy, wl.k, threads=1, lib=lib)
        if not np.allclose(r["scale"], ra["z"], rtol=1e-15, atol=0):
            fails.append("S* differs from the weighted mean of |z|")
        if not (np.array_equal(rn["scale"], r["scale"]) and np.array_equal(rn["z"], -r["z"])):
            fails.append("S* or Z not odd/even under z -> -z")
        if np.all(zz >= 0) and not np.allclose(r["scale"], r["z"], rtol=1e-15, atol=0):
            fails.append("S* differs from Z for z >= 0")

    for seed in range(2 if quick else 4):
        x, y, qx, qy = lattice_case(seed)
        for k in (1, 4, 9, 12):
            got, _ = oracle.knn(x, y, qx, qy, k, lib=lib)
            if not np.array_equal(got, brute_knn(x, y, qx, qy, k)):
                fails.append(f"knn lattice seed={seed} k={k} vs full sort")

    # Clark-Evans: uniform data, interior queries.
    rng = np.random.default_rng(7)
    n = 20000
    x, y = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    qx, qy = rng.uniform(0.15, 0.85, 3000), rng.uniform(0.15, 0.85, 3000)
    z = np.zeros(n)
    for k in (1, 10):
        R = oracle.interpolate(x, y, z, 1.0, qx, qy, k, lib=lib)["R"]
        se = R.std() / math.sqrt(len(R))
        if abs(R.mean() - clark_evans_mean_R(k)) > 5 * se + 0.002:
            fails.append(f"Clark-Evans k={k}: mean R {R.mean()} vs {clark_evans_mean_R(k)}")
    return fails


# ---------------------------------------------------------------------------------------------
# Tests
# ---------------------------------------------------------------------------------------------

def test_oracle_builds():
    assert os.path.exists(oracle.build())


def test_all_pins_pass():
    assert pin_failures() == []


@pytest.mark.parametrize("seed", range(3))
def test_knn_matches_printed_procedure(seed):
    x, y, qx, qy = lattice_case(100 + seed, n_side=8, m=25)
    for k in (1, 3, 8, 16):
        got, d2 = oracle.knn(x, y, qx, qy, k)
        assert np.array_equal(got, printed_knn_procedure(x, y, qx, qy, k))
        assert np.all(np.diff(d2, axis=1) >= 0)


def test_knn_random_float_inputs():
    wl = workloads.small_case(3, 700, 90, pattern="clustered")
    for k in (1, 10, 33):
        got, _ = oracle.knn(wl.x, wl.y, wl.qx, wl.qy, k)
        assert np.array_equal(got, brute_knn(wl.x, wl.y, wl.qx, wl.qy, k))


def test_knn_k_equals_n():
    wl = workloads.small_case(4, 17, 5)
    got, _ = oracle.knn(wl.x, wl.y, wl.qx, wl.qy, 17)
    assert np.array_equal(got, brute_knn(wl.x, wl.y, wl.qx, wl.qy, 17))


@pytest.mark.parametrize("pattern", ["uniform", "clustered"])
def test_weighted_mean_invariants(pattern):
    wl = workloads.small_case(11, 600, 150, pattern=pattern, levels=(0.5, 1.0, 2.0, 3.5, 6.0))
    r = oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx, wl.qy, wl.k, wl.levels)
    # alpha stays within the levels; Z is a convex combination of z.
    assert np.all(r["alpha"] >= 0.5 - 1e-15) and np.all(r["alpha"] <= 6.0 + 1e-15)
    assert np.all(r["z"] >= wl.z.min() - 1e-12) and np.all(r["z"] <= wl.z.max() + 1e-12)
    assert np.all(r["scale"] >= np.abs(r["z"]) * (1 - 1e-14))
    # Constant z is reproduced.
    c = oracle.interpolate(wl.x, wl.y, np.full(wl.n, 3.25), wl.area, wl.qx, wl.qy, wl.k,
                           wl.levels)
    assert np.allclose(c["z"], 3.25, rtol=1e-15, atol=0)
    # Permuting the data points changes nothing but the kNN index labels.
    perm = np.random.default_rng(5).permutation(wl.n)
    p = oracle.interpolate(wl.x[perm], wl.y[perm], wl.z[perm], wl.area, wl.qx, wl.qy, wl.k,
                           wl.levels)
    assert np.allclose(p["z"], r["z"], rtol=1e-13, atol=1e-13)
    assert np.allclose(p["alpha"], r["alpha"], rtol=1e-14)
    assert np.array_equal(np.sort(perm[p["knn"]], axis=1), np.sort(r["knn"], axis=1))
    # Exact binary scaling of coordinates by 2 (area by 4) leaves R, alpha and Z unchanged.
    s = oracle.interpolate(2 * wl.x, 2 * wl.y, wl.z, 4 * wl.area, 2 * wl.qx, 2 * wl.qy, wl.k,
                           wl.levels)
    assert np.array_equal(s["R"], r["R"]) and np.array_equal(s["alpha"], r["alpha"])
    assert np.allclose(s["z"], r["z"], rtol=1e-13, atol=1e-13)
    # Translation leaves the result unchanged up to input rounding.
    t = oracle.interpolate(wl.x + 37.0, wl.y - 11.0, wl.z, wl.area, wl.qx + 37.0, wl.qy - 11.0,
                           wl.k, wl.levels)
    assert np.allclose(t["z"], r["z"], rtol=1e-9, atol=1e-9)


def test_query_on_data_point_returns_its_value():
    wl = workloads.small_case(12, 300, 10)
    pick = np.array([0, 17, 299])
    r = oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.x[pick], wl.y[pick], wl.k)
    assert np.array_equal(r["z"], wl.z[pick])
    assert np.array_equal(r["knn"][:, 0], pick)


def test_equal_levels_reduce_to_textbook_idw():
    """All five levels equal to p: Eq. 6 returns p whatever R is, and Eq. 1 is Shepard's IDW."""
    wl = workloads.small_case(13, 400, 60, pattern="clustered")
    for p in (1.0, 2.0, 3.7):
        r = oracle.interpolate(wl.x, wl.y, wl.z, wl.area, wl.qx, wl.qy, 7, (p,) * 5)
        d = np.hypot(wl.qx[:, None] - wl.x[None, :], wl.qy[:, None] - wl.y[None, :])
        w = d ** (-p)
        ref = (w * wl.z).sum(1) / w.sum(1)
        assert np.allclose(r["z"], ref, rtol=1e-12, atol=1e-12)
        assert np.allclose(oracle.idw(wl.x, wl.y, wl.z, wl.qx, wl.qy, p)["z"], ref, rtol=1e-12,
                           atol=1e-12)


def test_alpha_mapping_is_continuous():
    """Eq. 6's segments meet at their ends, Eq. 5 is continuous for R_min = 0."""
    lv = (1.5, 4.0, 2.0, 7.0, 3.0)
    for b in (0.1, 0.3, 0.5, 0.7, 0.9):
        lo, hi = oracle.alpha_of_mu(b - 1e-12, lv), oracle.alpha_of_mu(b + 1e-12, lv)
        assert abs(lo - hi) < 1e-9
    for b in (0.0, 2.0):
        assert abs(oracle.mu_of_R(b - 1e-12) - oracle.mu_of_R(b + 1e-12)) < 1e-9


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.interpolate([0, 1], [0, 1], [0, 1], 1.0, [0.5], [0.5], 3)
    with pytest.raises(ValueError):
        oracle.interpolate([0, 1], [0, 1], [0, 1], 0.0, [0.5], [0.5], 1)
    with pytest.raises(ValueError):
        oracle.interpolate([0, 1], [0, 1], [0, 1], 1.0, [0.5], [0.5], 1, r_min=2.0, r_max=1.0)


# Each entry plants one plausible mistake into a copy of the oracle source.
MUTANTS = {
    "r_exp_no_factor_2": ("return 1.0 / (2.0 * sqrt(density));", "return 1.0 / sqrt(density);"),
    "r_exp_inverted": ("double density = (double)n / area;", "double density = area / (double)n;"),
    "mu_cos_sign": ("return 0.5 - 0.5 * cos(", "return 0.5 + 0.5 * cos("),
    "mu_shift_sign": ("* (R - r_min));", "* (R + r_min));"),
    "mu_range_divisor": ("(M_PI / r_max)", "(M_PI / (r_max - r_min))"),
    "alpha_seg2_swap": ("return 5.0 * a3 * (mu - 0.3) + a2 * (1.0 - 5.0 * (mu - 0.3));",
                        "return 5.0 * a2 * (mu - 0.3) + a3 * (1.0 - 5.0 * (mu - 0.3));"),
    "alpha_seg4_bound": ("if (mu <= 0.9)", "if (mu <= 0.8)"),
    "knn_ties_to_later": ("if (!(v < d2[k - 1]))", "if (!(v <= d2[k - 1]))"),
    "knn_sink_nonstrict": ("while (p > 0 && v < d2[p - 1]) {\n            d2[p] = d2[p - 1];\n"
                           "            idx[p] = idx[p - 1];\n            --p;\n        }\n"
                           "        d2[p] = v;\n        idx[p] = i;",
                           "while (p > 0 && v <= d2[p - 1]) {\n            d2[p] = d2[p - 1];\n"
                           "            idx[p] = idx[p - 1];\n            --p;\n        }\n"
                           "        d2[p] = v;\n        idx[p] = i;"),
    "r_obs_squared": ("s += sqrt(d2[j]);", "s += d2[j];"),
    "r_obs_sum_not_mean": ("double r_obs = s / (double)k;", "double r_obs = s;"),
    "weight_on_d2": ("pow(sqrt(dd), -alpha)", "pow(dd, -alpha)"),
    "weight_positive_power": ("pow(sqrt(dd), -alpha)", "pow(sqrt(dd), alpha)"),
    "phase2_first_k_only": ("for (int64_t i = 0; i < w->n; ++i) {\n            double dd",
                            "for (int64_t i = 0; i < w->k; ++i) {\n            double dd"),
    "dist_transposed": ("return dx * dx + dy * dy;", "return dx * dx + dx * dy;"),
    "coincident_first_only": ("Z = (sz0 + cz0) / (double)n0;", "Z = (sz0 + cz0);"),
    "scale_not_normalised": ("scale = (swa + cwa) / W;", "scale = (swa + cwa);"),
    "scale_signed": ("neumaier_add(&swa, &cwa, wi * fabs(w->z[i]));",
                     "neumaier_add(&swa, &cwa, wi * w->z[i]);"),
    "scale_coincident_sum": ("scale = (sa0 + ca0) / (double)n0;", "scale = (sa0 + ca0);"),
    "scale_coincident_signed": ("neumaier_add(&sa0, &ca0, fabs(w->z[i]));",
                                "neumaier_add(&sa0, &ca0, w->z[i]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.build()), "..", "aidw_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mut.c"
    c_path.write_text(mutated)
    so_path = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    str(c_path), "-o", str(so_path), "-lm"], check=True)
    lib = oracle.load_library(str(so_path))
    assert pin_failures(lib, quick=True), f"planted mistake {name} went unnoticed"
    shutil.rmtree(tmp_path, ignore_errors=True)
