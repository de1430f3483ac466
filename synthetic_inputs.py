"""Seeded synthetic inputs: point sets, right-hand sides and named workloads.

This module is shared by the tests, the CPU oracle checks and ``bench.py``. It holds
no H^2 arithmetic at all: it only draws points and vectors from fixed seeds and names
the workload parameters. The paper's test matrices are synthetic too (Sec. 6.1: a
2D grid with an exponential kernel, a 3D point set with an exponential kernel), so
nothing here stands in for a dataset.

Conventions
-----------
* Points are an ``(n, dim)`` float64 array, C order (row ``i`` = point ``i``).
* Multivectors are ``(n, nv)`` float64 arrays in Fortran order, i.e. column-major
  with leading dimension ``n`` (vector ``v`` occupies ``data[v*n:(v+1)*n]``).
* Kernels are named by ``(name, a, b, deg)``: ``"exp"`` = exp(-r/a),
  ``"gauss"`` = exp(-r^2/a), ``"imq"`` = (r^2+a)^(-b),
  ``"poly"`` = prod_d (1 + x_d y_d)^deg.
"""
from __future__ import annotations

import dataclasses
import numpy as np


def grid_2d(n_side: int) -> np.ndarray:
    """Uniform ``n_side x n_side`` grid on [0,1]^2, nodes at i/(n_side-1), x fastest."""
    if n_side < 2:
        raise ValueError("n_side must be >= 2")
    c = np.arange(n_side, dtype=np.float64) / float(n_side - 1)
    xs = np.tile(c, n_side)
    ys = np.repeat(c, n_side)
    return np.ascontiguousarray(np.stack([xs, ys], axis=1))


def grid_3d(n_side: int) -> np.ndarray:
    """Uniform ``n_side^3`` grid on [0,1]^3, nodes at i/(n_side-1), x fastest then y."""
    c = np.arange(n_side, dtype=np.float64) / float(n_side - 1)
    xs = np.tile(c, n_side * n_side)
    ys = np.tile(np.repeat(c, n_side), n_side)
    zs = np.repeat(c, n_side * n_side)
    return np.ascontiguousarray(np.stack([xs, ys, zs], axis=1))


def uniform_cloud(n: int, dim: int, seed: int) -> np.ndarray:
    """``n`` points uniform in [0,1]^dim from ``numpy.random.default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((n, dim)))


def gaussian_vectors(n: int, nv: int, seed: int) -> np.ndarray:
    """``(n, nv)`` column-major multivector with N(0,1) entries.

    Vector ``v`` is ``standard_normal(n*nv)[v*n:(v+1)*n]`` of ``default_rng(seed)``,
    so the first column does not depend on ``nv``.
    """
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(n * nv)
    return np.asfortranarray(flat.reshape(nv, n).T)


def uniform_vectors(n: int, nv: int, seed: int) -> np.ndarray:
    """``(n, nv)`` column-major multivector with U[0,1) entries (the Sec. 6.1 accuracy probe)."""
    rng = np.random.default_rng(seed)
    flat = rng.random(n * nv)
    return np.asfortranarray(flat.reshape(nv, n).T)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named operator + right-hand-side recipe."""

    name: str
    points: str            # "grid2d:<side>", "grid3d:<side>" or "cloud:<n>:<dim>:<seed>"
    kernel: tuple          # (name, a, b, deg)
    leaf_size: int
    cheb_order: int
    eta: float
    nv: int
    x_seed: int

    def make_points(self) -> np.ndarray:
        kind, *args = self.points.split(":")
        if kind == "grid2d":
            return grid_2d(int(args[0]))
        if kind == "grid3d":
            return grid_3d(int(args[0]))
        if kind == "cloud":
            return uniform_cloud(int(args[0]), int(args[1]), int(args[2]))
        raise ValueError(self.points)

    def make_x(self, n: int, nv: int | None = None) -> np.ndarray:
        return gaussian_vectors(n, self.nv if nv is None else nv, self.x_seed)


# The 2D spatial-statistics style set of Sec. 6.1 at N = 4096: 64x64 grid, exp(-r/0.1),
# leaf 64, 4x4 Chebyshev grid (rank 16), eta = 0.9. Small enough for dense checks.
GRID64_EXP = Workload("grid64_exp", "grid2d:64", ("exp", 0.1, 0.0, 0), 64, 4, 0.9, 1, 1)

# Memory-bound single-vector case: 1024x1024 grid (N = 2^20), Gaussian exp(-r^2/0.01),
# leaf 64, 8x8 Chebyshev grid (rank 64), eta = 0.7.
GRID1024_GAUSS = Workload("grid1024_gauss", "grid2d:1024", ("gauss", 0.01, 0.0, 0), 64, 8, 0.7, 1, 1)

# Multi-RHS case: 2^21 uniform points in [0,1]^3 (seed 0), exp(-r/0.2), leaf 64,
# 4x4x4 Chebyshev grid (rank 64), eta = 0.7, 32 Gaussian vectors (seed 1).
CLOUD3D_EXP = Workload("cloud3d_exp", "cloud:2097152:3:0", ("exp", 0.2, 0.0, 0), 64, 4, 0.7, 32, 1)


def grid_gauss(side: int) -> Workload:
    """The Gaussian grid workload at another grid side (same kernel, rank, eta)."""
    return dataclasses.replace(GRID1024_GAUSS, name=f"grid{side}_gauss", points=f"grid2d:{side}")


def cloud3d(n: int, nv: int = 32) -> Workload:
    """The 3D cloud workload at another size (same distribution, kernel, rank, eta)."""
    return dataclasses.replace(CLOUD3D_EXP, name=f"cloud3d_{n}", points=f"cloud:{n}:3:0", nv=nv)


# The algebraic-compression sets of Sec. 6 (matrix compression): a 2D grid with a 6x6
# Chebyshev grid (rank 36), exp(-r/0.1), leaf 64, eta 0.9 at N = 2^20; a 3D grid with
# tri-cubic interpolation (rank 64), exp(-r/0.2), leaf 64, eta 0.95 at N = 2^18 (64^3). Both
# are compressed to the relative tolerance COMPRESS_TAU.
COMPRESS_2D = Workload("compress_grid2d_exp", "grid2d:1024", ("exp", 0.1, 0.0, 0), 64, 6, 0.9, 1, 1)
COMPRESS_3D = Workload("compress_grid3d_exp", "grid3d:64", ("exp", 0.2, 0.0, 0), 64, 4, 0.95, 1, 1)
COMPRESS_TAU = 1e-3

WORKLOADS = {w.name: w for w in (GRID64_EXP, GRID1024_GAUSS, CLOUD3D_EXP, COMPRESS_2D, COMPRESS_3D)}


@dataclasses.dataclass(frozen=True)
class BatchMember:
    """One operator of the batched workload: its points, kernel, construction parameters
    and the number of vectors of its product."""
    name: str
    points: np.ndarray
    kernel: tuple
    leaf_size: int
    cheb_order: int
    eta: float
    nv: int
    x_seed: int

    def make_x(self) -> np.ndarray:
        return gaussian_vectors(len(self.points), self.nv, self.x_seed)


def uneven_batch(count: int = 64, n_min: int = 2 ** 12, n_max: int = 2 ** 18, seed: int = 4,
                 nv_max: int = 16) -> list:
    """Operators of uneven size for a batched product, drawn from default_rng(seed) in order:
    N log-uniform in [n_min, n_max]; even members are 2D grids with side round(sqrt(N))
    (N := side^2) and a Chebyshev order in {4, ..., 8} per dimension, odd members uniform 3D
    clouds with an order in {3, 4}; kernel exp(-r/l) with l uniform in [0.05, 0.3]; leaf 64,
    eta 0.7; nv uniform in {1, ..., nv_max}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))))
        ell = float(rng.uniform(0.05, 0.3))
        nv = int(rng.integers(1, nv_max + 1))
        if i % 2 == 0:
            side = max(2, int(round(np.sqrt(n))))
            p = int(rng.integers(4, 9))
            pts = grid_2d(side)
            name = f"grid{side}"
        else:
            p = int(rng.integers(3, 5))
            pts = uniform_cloud(n, 3, int(rng.integers(0, 2 ** 31)))
            name = f"cloud3d_{n}"
        out.append(BatchMember(f"{i:02d}_{name}", pts, ("exp", ell, 0.0, 0), 64, p, 0.7, nv, 10_000 + i))
    return out
