"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module only draws random numbers and lays out point sets.  It holds none
of the method's arithmetic (no kernel evaluation, no factorization), so both the
GPU path and the CPU oracle may import it without sharing any of the method.

Workloads (scattered 2-D locations standing in for the paper's ICOADS set,
Sec. 5.4, which is not available here):

* ``uniform(n, seed)``: i.i.d. U[0,1]^2.
* ``mixture(n, seed)``: half U[0,1]^2, half from four isotropic Gaussian
  clusters (sigma 0.03) whose centres are drawn once from U[0.2,0.8]^2 with
  seed 12345; cluster points falling outside [0,1]^2 are redrawn.
* ``grid(side, lo, hi)``: the regular sqrt(n) x sqrt(n) grid of Sec. 5.1.

All draws use NumPy's PCG64 generator so that a seed fixes the data exactly.
"""
from __future__ import annotations

import numpy as np

CLUSTER_SEED = 12345
CLUSTER_SIGMA = 0.03
N_CLUSTERS = 4


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in the unit square, shape (n, 2), float64."""
    return _rng(seed).random((n, 2))


def cluster_centres() -> np.ndarray:
    """The four fixed cluster centres of the mixture workload, shape (4, 2)."""
    return 0.2 + 0.6 * _rng(CLUSTER_SEED).random((N_CLUSTERS, 2))


def mixture(n: int, seed: int) -> np.ndarray:
    """Uniform + 4-cluster mixture: n//2 uniform points, the rest split evenly
    over the four clusters (the last cluster takes the remainder)."""
    rng = _rng(seed)
    n_uni = n // 2
    pts = [rng.random((n_uni, 2))]
    centres = cluster_centres()
    n_cl = n - n_uni
    per = [n_cl // N_CLUSTERS] * N_CLUSTERS
    per[-1] += n_cl - sum(per)
    for c, m in zip(centres, per):
        got = np.empty((0, 2))
        while got.shape[0] < m:
            draw = c + CLUSTER_SIGMA * rng.standard_normal((m - got.shape[0], 2))
            keep = np.all((draw >= 0.0) & (draw <= 1.0), axis=1)
            got = np.vstack([got, draw[keep]])
        pts.append(got)
    return np.ascontiguousarray(np.vstack(pts))


def grid(side: int, lo: float = 0.0, hi: float = 100.0) -> np.ndarray:
    """side x side regular grid discretizing [lo, hi]^2 (Sec. 5.1), (n, 2)."""
    t = lo + (hi - lo) * (np.arange(side) + 0.5) / side
    gx, gy = np.meshgrid(t, t, indexing="xy")
    return np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel()], axis=1))


def standard_normal(n: int, seed: int, ncols: int | None = None) -> np.ndarray:
    """N(0,1) draws: shape (n,) or (n, ncols)."""
    rng = _rng(seed)
    return rng.standard_normal(n if ncols is None else (n, ncols))


def subsample(points: np.ndarray, m: int, seed: int) -> np.ndarray:
    """m distinct rows of ``points`` chosen uniformly without replacement."""
    idx = np.sort(_rng(seed).choice(points.shape[0], size=m, replace=False))
    return np.ascontiguousarray(points[idx]), idx


# Workload descriptions (sizes, kernel, theta, tolerances, seeds).
MATERN12, MATERN32, MATERN52, MATERN1, RQ = 0, 1, 2, 3, 4

WORKLOADS = {
    "matern32_uniform_n4096": dict(
        n=4096, points="uniform", seed_points=1, seed_z=2, family=MATERN32,
        alpha=0.0, theta=(0.1, 1.0, 1e-2), tol_fact=1e-9, tol_peel=1e-6),
    "matern32_mixture_n262144": dict(
        n=262144, points="mixture", seed_points=3, seed_z=5, seed_w=6,
        family=MATERN32, alpha=0.0, theta=(0.05, 2.0, 1e-2), tol_fact=1e-9,
        tol_peel=1e-6, subsample=16384, seed_subsample=4),
    "rq2_uniform_n1048576": dict(
        n=1048576, points="uniform", seed_points=7, seed_z=8, family=RQ,
        alpha=2.0, theta=(0.02, 1.0, 1e-2), tol_fact=1e-9, tol_peel=1e-6),
    # the paper's gridded experiments (Sec. 5.1, 5.3): sqrt(n) x sqrt(n) grid
    # of [0, 100]^2, anisotropic theta = [10, 7] as (l1, s2, nug, l2) with unit
    # variance and noise 1e-4, eps_fact = eps_peel / 1000
    "matern32_grid_aniso_n262144": dict(
        n=262144, points="grid", seed_points=0, seed_z=11, family=MATERN32,
        alpha=0.0, theta=(10.0, 1.0, 1e-4, 7.0), tol_fact=1e-9, tol_peel=1e-6),
    "rq_half_grid_aniso_n262144": dict(
        n=262144, points="grid", seed_points=0, seed_z=12, family=RQ,
        alpha=0.5, theta=(10.0, 1.0, 1e-4, 7.0), tol_fact=1e-9, tol_peel=1e-6),
}


def make_points(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform(n, seed)
    if kind == "mixture":
        return mixture(n, seed)
    if kind == "grid":
        side = int(round(n ** 0.5))
        if side * side != n:
            raise ValueError("a grid workload needs a square point count")
        return grid(side)
    raise ValueError(f"unknown point distribution {kind!r}")
