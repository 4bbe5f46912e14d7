"""Seeded synthetic inputs for AIDW, shared by the tests, the benchmark and the smoke check.

This module only draws points and values; it holds none of the method's arithmetic. The paper
(Sec. 4) measures on points "randomly created within a square" with as many queries as data
points; it names no dataset, so every workload here is synthetic:

* ``uniform_unit``   -- 1,024 x 1,024 uniform points in the unit square, A = 1,
                        z = sin(3x) cos(2y) + 0.01 N(0,1), k = 10.
* ``uniform_paper``  -- 1,048,576 x 1,048,576 uniform points in [0,1000]^2, A = 1e6,
                        z = sin(x/100) + cos(y/150) + 0.05 N(0,1), k = 10 (the paper's largest
                        size class, rounded to a power of two).
* ``clustered_grid`` -- 2,097,152 data points: 90 % from 32 Gaussian clusters (sigma log-uniform
                        in [5, 50]) and 10 % uniform background over [0,1000]^2, redrawn when
                        outside; 1448 x 1448 queries at grid-cell centres; z ~ lognormal(0,1).
* ``batched``        -- many independent datasets of log-uniform sizes, uniform or clustered.
* ``served``         -- resident datasets plus a Poisson stream of query requests.

All draws come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEFAULT_LEVELS = (1.0, 2.0, 3.0, 4.0, 5.0)


@dataclasses.dataclass
class Workload:
    """One AIDW problem: data points, values, study area, queries and parameters."""

    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    area: float
    qx: np.ndarray
    qy: np.ndarray
    k: int = 10
    levels: tuple = DEFAULT_LEVELS
    r_min: float = 0.0
    r_max: float = 2.0

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def m(self) -> int:
        return int(self.qx.shape[0])

    def as_f32(self) -> "Workload":
        """The same problem with every coordinate and value rounded to float32 and widened
        back to float64: the exact inputs a float32 path sees."""
        r = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
        return dataclasses.replace(self, x=r(self.x), y=r(self.y), z=r(self.z),
                                   qx=r(self.qx), qy=r(self.qy))

    def query_subset(self, idx: np.ndarray) -> "Workload":
        return dataclasses.replace(self, qx=self.qx[idx].copy(), qy=self.qy[idx].copy())


def _uniform(rng, n, lo, hi):
    return rng.uniform(lo, hi, n), rng.uniform(lo, hi, n)


def clustered_points(rng, n: int, side: float, n_clusters: int, sigma_lo: float,
                     sigma_hi: float, background: float = 0.1, x0: float = 0.0,
                     y0: float = 0.0):
    """n points in [x0, x0+side] x [y0, y0+side]: a fraction ``background`` uniform, the rest
    from ``n_clusters`` equally weighted isotropic Gaussians with centres uniform in the square
    and sigma log-uniform in [sigma_lo, sigma_hi]; samples outside the square are redrawn."""
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    cx = rng.uniform(0.0, side, n_clusters)
    cy = rng.uniform(0.0, side, n_clusters)
    sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_clusters))
    comp = rng.integers(0, n_clusters, n_cl)
    px = cx[comp] + sig[comp] * rng.standard_normal(n_cl)
    py = cy[comp] + sig[comp] * rng.standard_normal(n_cl)
    bad = (px < 0) | (px > side) | (py < 0) | (py > side)
    while bad.any():
        nb = int(bad.sum())
        c = comp[bad]
        px[bad] = cx[c] + sig[c] * rng.standard_normal(nb)
        py[bad] = cy[c] + sig[c] * rng.standard_normal(nb)
        bad = (px < 0) | (px > side) | (py < 0) | (py > side)
    bx, by = _uniform(rng, n_bg, 0.0, side)
    x = np.concatenate([px, bx])
    y = np.concatenate([py, by])
    perm = rng.permutation(n)
    return x[perm] + x0, y[perm] + y0


def smooth_values(rng, x, y, side: float, noise: float = 0.05):
    """z = sin(x / (0.1 side)) + cos(y / (0.15 side)) + noise * N(0,1)."""
    return (np.sin(x / (side * 0.1)) + np.cos(y / (side * 0.15))
            + noise * rng.standard_normal(x.shape[0]))


def uniform_unit(seed: int = 0, n: int = 1024, m: int = 1024, k: int = 10) -> Workload:
    rng = np.random.default_rng(seed)
    x, y = _uniform(rng, n, 0.0, 1.0)
    z = np.sin(3.0 * x) * np.cos(2.0 * y) + 0.01 * rng.standard_normal(n)
    qx, qy = _uniform(rng, m, 0.0, 1.0)
    return Workload("uniform_unit", x, y, z, 1.0, qx, qy, k=k)


def uniform_paper(seed: int = 0, n: int = 1 << 20, m: int = 1 << 20, k: int = 10,
                  side: float = 1000.0) -> Workload:
    rng = np.random.default_rng(seed)
    x, y = _uniform(rng, n, 0.0, side)
    z = np.sin(x / 100.0) + np.cos(y / 150.0) + 0.05 * rng.standard_normal(n)
    qx, qy = _uniform(rng, m, 0.0, side)
    return Workload("uniform_paper", x, y, z, side * side, qx, qy, k=k)


def clustered_grid(seed: int = 0, n: int = 1 << 21, grid: int = 1448, k: int = 10,
                   side: float = 1000.0) -> Workload:
    rng = np.random.default_rng(seed)
    x, y = clustered_points(rng, n, side, 32, 5.0, 50.0, 0.1)
    z = rng.lognormal(0.0, 1.0, n)
    c = (np.arange(grid) + 0.5) * (side / grid)
    qy, qx = np.meshgrid(c, c, indexing="ij")
    return Workload("clustered_grid", x, y, z, side * side, qx.ravel().copy(),
                    qy.ravel().copy(), k=k)


def small_case(seed: int, n: int, m: int, k: int = 10, pattern: str = "uniform",
               side: float = 100.0, levels=DEFAULT_LEVELS) -> Workload:
    """A parity case of any size: uniform or clustered data, queries uniform in the square,
    z = smooth field plus noise."""
    rng = np.random.default_rng(seed)
    if pattern == "uniform":
        x, y = _uniform(rng, n, 0.0, side)
    else:
        ncl = int(rng.integers(4, 33))
        x, y = clustered_points(rng, n, side, ncl, 0.005 * side, 0.05 * side, 0.1)
    z = smooth_values(rng, x, y, side)
    qx, qy = _uniform(rng, m, 0.0, side)
    return Workload(f"{pattern}_{n}x{m}", x, y, z, side * side, qx, qy, k=k,
                    levels=tuple(levels))


def batched(seed: int = 0, count: int = 256, n_lo: int = 1024, n_hi: int = 262144,
            m_lo: int = 1024, m_hi: int = 65536, ks=(6, 10, 15)) -> list[Workload]:
    """Independent datasets for one batched launch: n and m log-uniform, region side
    log-uniform in [10, 1000], uniform or clustered pattern with equal odds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        side = float(math.exp(rng.uniform(math.log(10.0), math.log(1000.0))))
        k = int(rng.choice(ks))
        if rng.uniform() < 0.5:
            x, y = _uniform(rng, n, 0.0, side)
            pat = "uniform"
        else:
            x, y = clustered_points(rng, n, side, int(rng.integers(4, 33)), 0.005 * side,
                                    0.05 * side, 0.1)
            pat = "clustered"
        z = smooth_values(rng, x, y, side)
        qx, qy = _uniform(rng, m, 0.0, side)
        out.append(Workload(f"batch{i}_{pat}", x, y, z, side * side, qx, qy, k=k))
    return out


def served_datasets(seed: int = 0, count: int = 64, n_lo: int = 16384,
                    n_hi: int = 1 << 20) -> list[Workload]:
    """Resident datasets for the serving loop (queries come from ``served_requests``)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        side = float(math.exp(rng.uniform(math.log(10.0), math.log(1000.0))))
        if rng.uniform() < 0.5:
            x, y = _uniform(rng, n, 0.0, side)
        else:
            x, y = clustered_points(rng, n, side, int(rng.integers(4, 33)), 0.005 * side,
                                    0.05 * side, 0.1)
        z = smooth_values(rng, x, y, side)
        e = np.empty(0)
        out.append(Workload(f"served{i}", x, y, z, side * side, e, e, k=10))
    return out


def served_requests(datasets: list[Workload], seed: int = 1, rate: float = 2000.0,
                    duration_s: float = 10.0, m_lo: int = 256, m_hi: int = 262144):
    """Poisson arrivals: list of (arrival_time_s, dataset_index, qx, qy)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        d = int(rng.integers(0, len(datasets)))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        side = math.sqrt(datasets[d].area)
        qx = rng.uniform(0.0, side, m)
        qy = rng.uniform(0.0, side, m)
        out.append((t, d, qx, qy))
    return out


def served_arrivals(datasets: list[Workload], seed: int = 1, rate: float = 2000.0,
                    duration_s: float = 10.0, m_lo: int = 256, m_hi: int = 262144):
    """Poisson arrivals without their query arrays: list of (arrival_time_s, dataset_index,
    query_count), query counts log-uniform in [m_lo, m_hi]. The queries come from
    ``served_query_pool`` (long runs would not fit in host memory with one array per
    request)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        d = int(rng.integers(0, len(datasets)))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        out.append((t, d, m))
    return out


def served_query_pool(datasets: list[Workload], seed: int = 2, size: int = 262144):
    """Per dataset, `size` float32 query points uniform in its square; a request of m queries
    takes a contiguous slice of its dataset's pool."""
    rng = np.random.default_rng(seed)
    out = []
    for w in datasets:
        side = math.sqrt(w.area)
        out.append((rng.uniform(0.0, side, size).astype(np.float32),
                    rng.uniform(0.0, side, size).astype(np.float32)))
    return out
