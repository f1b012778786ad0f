"""Seeded synthetic TSP instances (integer EUC_2D coordinates).

This module holds no arithmetic of the method itself; both the GPU library's
tests and the CPU oracle draw their inputs from here.

* ``uniform(n, seed, side)``: points uniform in [0, side)^2 (the paper's
  random-uniform and TSPLIB-like settings).
* ``stippled(n, seed, blobs, ridges, side)``: stand-in for the "TSP Art"
  instances of the paper's large-instance study (Sec. 5.4.2, Table 4), which
  are stippled images and are not shipped here.  Density on a 1024^2 grid is a
  sum of isotropic Gaussian blobs (uniform centres, sigma log-uniform in
  [0.005, 0.06] of the side, amplitude U[0.3, 1]) plus smooth cubic Bezier
  ridges of width 0.003 of the side, plus a 5 % uniform floor; grid cells are
  sampled by that density with uniform jitter inside the cell.  Only the shape
  (clustered density, smooth curves) is imitated.
* ``batch_sizes(count, seed, lo, hi)``: n log-uniform in [lo, hi].

All generators use ``numpy.random.Generator(Philox(seed))`` and resample
duplicate points, so every pair of distinct nodes has a positive distance.
"""
from __future__ import annotations

import numpy as np

GRID = 1024


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _dedupe(xy: np.ndarray, side: int, redraw) -> np.ndarray:
    """Replace repeated points by fresh draws until all points are distinct."""
    for _ in range(1000):
        key = xy[:, 0].astype(np.int64) * side + xy[:, 1]
        _, first = np.unique(key, return_index=True)
        dup = np.ones(len(xy), bool)
        dup[first] = False
        if not dup.any():
            return xy
        xy[dup] = redraw(int(dup.sum()))
    raise RuntimeError("could not draw distinct points")


def uniform(n: int, seed: int = 1001, side: int = 1_000_000) -> np.ndarray:
    """n distinct integer points uniform in [0, side)^2, shape (n, 2) int32."""
    if n > side * side:
        raise ValueError("more points than lattice sites")
    rng = _rng(seed)

    def draw(m):
        return rng.integers(0, side, size=(m, 2), dtype=np.int64)

    return np.ascontiguousarray(_dedupe(draw(n), side, draw).astype(np.int32))


def _density(rng: np.random.Generator, blobs: int, ridges: int) -> np.ndarray:
    g = (np.arange(GRID) + 0.5) / GRID
    dens = np.zeros((GRID, GRID), np.float64)
    cx = rng.random(blobs)
    cy = rng.random(blobs)
    sig = np.exp(rng.uniform(np.log(0.005), np.log(0.06), blobs))
    amp = rng.uniform(0.3, 1.0, blobs)
    for i in range(blobs):
        gx = np.exp(-0.5 * ((g - cx[i]) / sig[i]) ** 2)
        gy = np.exp(-0.5 * ((g - cy[i]) / sig[i]) ** 2)
        dens += amp[i] * np.outer(gx, gy)
    width = 0.003
    half = int(np.ceil(4 * width * GRID)) + 1
    for _ in range(ridges):
        ctrl = rng.uniform(0.1, 0.9, size=(4, 2))
        amp_r = rng.uniform(0.3, 1.0)
        t = np.linspace(0.0, 1.0, 4000)[:, None]
        pts = ((1 - t) ** 3 * ctrl[0] + 3 * (1 - t) ** 2 * t * ctrl[1]
               + 3 * (1 - t) * t ** 2 * ctrl[2] + t ** 3 * ctrl[3])
        for px, py in pts[::4]:
            ix, iy = int(px * GRID), int(py * GRID)
            x0, x1 = max(ix - half, 0), min(ix + half + 1, GRID)
            y0, y1 = max(iy - half, 0), min(iy + half + 1, GRID)
            wx = np.exp(-0.5 * ((g[x0:x1] - px) / width) ** 2)
            wy = np.exp(-0.5 * ((g[y0:y1] - py) / width) ** 2)
            dens[x0:x1, y0:y1] += amp_r * 0.05 * np.outer(wx, wy)
    dens /= dens.sum()
    return 0.95 * dens + 0.05 / (GRID * GRID)


def stippled(n: int, seed: int = 2002, blobs: int = 64, ridges: int = 8,
             side: int = 100_000) -> np.ndarray:
    """n distinct clustered integer points in [0, side)^2, shape (n, 2) int32."""
    if n > side * side:
        raise ValueError("more points than lattice sites")
    rng = _rng(seed)
    p = _density(rng, blobs, ridges).reshape(-1)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    cell = side / GRID

    def draw(m):
        c = np.searchsorted(cdf, rng.random(m), side="right")
        c = np.minimum(c, GRID * GRID - 1)
        ix, iy = c // GRID, c % GRID
        x = np.floor((ix + rng.random(m)) * cell).astype(np.int64)
        y = np.floor((iy + rng.random(m)) * cell).astype(np.int64)
        return np.stack([np.clip(x, 0, side - 1), np.clip(y, 0, side - 1)], axis=1)

    return np.ascontiguousarray(_dedupe(draw(n), side, draw).astype(np.int32))


def batch_sizes(count: int, seed: int = 4000, lo: int = 200, hi: int = 20_000) -> np.ndarray:
    """Instance sizes log-uniform in [lo, hi] (rounded), shape (count,) int32."""
    rng = _rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int32)


def batch_instances(count: int, seed: int = 4000, lo: int = 200, hi: int = 20_000,
                    side: int = 1_000_000) -> list:
    """`count` independent uniform instances with log-uniform sizes in [lo, hi];
    instance i is uniform(n_i, seed * 1000 + i + 1, side)."""
    sizes = batch_sizes(count, seed, lo, hi)
    return [uniform(int(n), seed=seed * 1000 + i + 1, side=side) for i, n in enumerate(sizes)]


def lattice(rows: int, cols: int, step: int = 10) -> np.ndarray:
    """Regular grid: maximal distance ties (edge case for neighbour order)."""
    y, x = np.divmod(np.arange(rows * cols), cols)
    return np.ascontiguousarray(np.stack([x * step, y * step], axis=1).astype(np.int32))


# The five workloads of the study: the three plain colonies are listed here.
WORKLOADS = {
    "uniform1k": dict(kind="uniform", n=1_000, seed=1001, side=1_000_000, ants=32, iters=200),
    "stippled100k": dict(kind="stippled", n=100_000, seed=2002, blobs=64, ridges=8,
                         side=100_000, ants=1024, iters=100),
    "stippled200k": dict(kind="stippled", n=200_000, seed=3003, blobs=256, ridges=16,
                         side=100_000, ants=2048, iters=50),
}


# The batched workload: independent uniform instances run together; colony i
# uses Philox seed seed0 + i.
BATCH_WORKLOADS = {
    "batch512": dict(count=512, seed=4000, lo=200, hi=20_000, side=1_000_000, k=16, ants=64, iters=100,
                     seed0=1),
}


# The served workload: a Poisson stream of uniform instances with log-uniform
# sizes; request i uses Philox seed seed0 + i.
SERVE_WORKLOADS = {
    "serve100k": dict(seed=5000, lo=1_000, hi=100_000, side=1_000_000, k=16, ants=256, iters=50, seed0=1),
}


def serve_trace(name: str, count: int, rate: float, seed: int = 0):
    """(instances, seeds, arrival offsets in seconds) of `count` requests of a
    served workload arriving as a Poisson process of `rate` per second."""
    w = SERVE_WORKLOADS[name]
    xs = batch_instances(count, w["seed"] + seed, w["lo"], w["hi"], w["side"])
    gaps = _rng(w["seed"] + 7919 + seed).exponential(1.0 / rate, count)
    gaps[0] = 0.0
    return xs, np.arange(w["seed0"], w["seed0"] + count, dtype=np.uint64), np.cumsum(gaps)


def batch_workload(name: str):
    """(instances, seeds) of a batched workload."""
    w = BATCH_WORKLOADS[name]
    xs = batch_instances(w["count"], w["seed"], w["lo"], w["hi"], w["side"])
    return xs, np.arange(w["seed0"], w["seed0"] + w["count"], dtype=np.uint64)


def workload_points(name: str) -> np.ndarray:
    w = WORKLOADS[name]
    if w["kind"] == "uniform":
        return uniform(w["n"], w["seed"], w["side"])
    return stippled(w["n"], w["seed"], w["blobs"], w["ridges"], w["side"])
