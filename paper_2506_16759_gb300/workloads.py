"""Seeded synthetic inputs for the H2 construction workloads.

This module only draws random numbers and lays out point sets; it holds none
of the construction's arithmetic.  Both the CPU oracle (tests) and the CUDA
path take their inputs from here, so the two sides see identical bits.

Workloads (the paper's test problems are synthetic point clouds, Sec. V-A):

* ``c1``  N=4096 points uniform in [0,1]^2, exponential kernel exp(-r/0.2)
          plus 1e-4 on the diagonal, leaf 64, eta 0.7, tol 1e-6, dense sketch.
* ``c2``  N=131072 points uniform in [0,1]^3, Matern-3/2 with l=0.1 plus a
          1e-4 nugget, leaf 64, eta 0.7, tol 1e-6, fused kernel-summation sketch.
* ``c3``  the 48^3 cell centres of a regular grid on [0,1]^3 (h=1/48),
          1/(4 pi r) off the diagonal and 0.3799 h^2 on it, leaf 64, eta 0.7,
          tol 1e-5, fused kernel-summation sketch.
* ``c4``  N=262144 points uniform in [0,1]^3; the operator is the sum of two
          prebuilt H2 matrices (exponential l=0.1 and Gaussian sigma=0.05).
* ``c5``  64 independent 2D/3D exponential covariance instances with N drawn
          log-uniform in [2048, 32768] and l uniform in [0.05, 0.3].

The two kernel problems exactly as the paper states them (Sec. V-A), both on
points uniform in the unit cube, sketched through the matvec of an H2 matrix
prebuilt for the same kernel (``paper_problem``):

* ``exp3d``      exp(-r/0.2), no nugget;
* ``helmholtz``  cos(3r)/r off the diagonal, 0 on it (the paper defines the
                 operator for x != y only);
* ``update``     the exp3d H2 matrix plus a symmetric rank-32 product U S U^T,
                 recompressed into one H2 matrix (entries from the operand's
                 representation plus the product's entries).

Every workload uses 32 initial Gaussian samples, increments of 16 and at most
256 samples.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kernel identifiers shared by the C ABI (h2_kernel) and the oracle.
K_EXP = 0
K_MATERN32 = 1
K_GAUSS = 2
K_LAPLACE_IE = 3
K_POLY = 4
K_H2SUM = 5
K_HELMHOLTZ_IE = 6

KERNEL_NAMES = {K_EXP: "exp", K_MATERN32: "matern32", K_GAUSS: "gauss",
                K_LAPLACE_IE: "laplace_ie", K_POLY: "poly", K_H2SUM: "h2sum",
                K_HELMHOLTZ_IE: "helmholtz_ie"}


@dataclass
class Workload:
    name: str
    n: int
    dim: int
    kernel: int
    params: tuple
    leaf_size: int = 64
    eta: float = 0.7
    tol: float = 1e-6
    d0: int = 32
    d_inc: int = 16
    d_max: int = 256
    sketch: str = "ksum"          # "dense", "ksum" or "h2sum"
    point_seed: int = 0
    omega_seed: int = 0
    grid: bool = False
    extra: dict = field(default_factory=dict)

    def points(self) -> np.ndarray:
        if self.grid:
            side = round(self.n ** (1.0 / self.dim))
            return grid_points(side, self.dim)
        return uniform_points(self.n, self.dim, self.point_seed)

    def omega(self, d: int | None = None) -> np.ndarray:
        return gaussian_omega(self.n, self.d_max if d is None else d, self.omega_seed)


def uniform_points(n: int, dim: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1]^dim, FP64, row-major (n, dim)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.random((n, dim)))


def grid_points(side: int, dim: int = 3) -> np.ndarray:
    """Cell centres ((i+1/2)h, ...) of a regular side^dim grid on [0,1]^dim."""
    h = 1.0 / side
    axes = [(np.arange(side, dtype=np.float64) + 0.5) * h for _ in range(dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([m.reshape(-1) for m in mesh], axis=1))


def gaussian_omega(n: int, d: int, seed: int) -> np.ndarray:
    """Gaussian N(0,1) test matrix, (n, d) FP64, rows in original point order.

    Returned column-major (Fortran order) so that column blocks are contiguous;
    column c is the c-th sample vector.  Draws are made column by column so the
    first d columns do not depend on how many columns are requested.
    """
    rng = np.random.default_rng(seed)
    cols = [rng.standard_normal(n) for _ in range(d)]
    if not cols:
        return np.zeros((n, 0), order="F")
    return np.asfortranarray(np.stack(cols, axis=1))


def gaussian_probe(n: int, d: int, seed: int) -> np.ndarray:
    """Gaussian probe block G (n, d) used by the randomized error estimator."""
    return gaussian_omega(n, d, seed + 7919)


def config(name: str) -> Workload:
    """The named workload (c1..c4; c5 is a list, see ``c5_instances``)."""
    if name == "c1":
        return Workload("c1", 4096, 2, K_EXP, (0.2, 1e-4), tol=1e-6, sketch="dense",
                        point_seed=1, omega_seed=2)
    if name == "c2":
        return Workload("c2", 131072, 3, K_MATERN32, (0.1, 1e-4), tol=1e-6, sketch="ksum",
                        point_seed=3, omega_seed=13)
    if name == "c3":
        h = 1.0 / 48.0
        return Workload("c3", 48 ** 3, 3, K_LAPLACE_IE, (0.3799 * h * h,), tol=1e-5,
                        sketch="ksum", grid=True, omega_seed=23)
    if name == "c4":
        return Workload("c4", 262144, 3, K_H2SUM, (), tol=1e-6, sketch="h2sum",
                        point_seed=4, omega_seed=33,
                        extra={"operands": [(K_EXP, (0.1, 0.0)), (K_GAUSS, (0.05, 0.0))],
                               "operand_tol": 1e-8})
    raise KeyError(name)


def scaled(w: Workload, n: int, name: str | None = None) -> Workload:
    """The same workload family at a different point count (same seeds)."""
    import dataclasses
    if w.grid:
        side = max(2, round(n ** (1.0 / w.dim)))
        n = side ** w.dim
    return dataclasses.replace(w, n=n, name=name or f"{w.name}@{n}")


def c5_instances(count: int = 64, seed: int = 5) -> list[Workload]:
    """Independent exponential-covariance instances of uneven size."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(2048.0), math.log(32768.0)))))
        ell = float(rng.uniform(0.05, 0.3))
        dim = int(rng.integers(2, 4))
        out.append(Workload(f"c5[{i}]", n, dim, K_EXP, (ell, 1e-4), tol=1e-6, sketch="ksum",
                            point_seed=1000 + i, omega_seed=2000 + i))
    return out


def low_rank_factors(n: int, r: int, seed: int, scale: float) -> tuple:
    """Factors (U, V) of a symmetric rank-r product U V^T = U S U^T: U has
    i.i.d. N(0, 1/n) entries, S = diag(s) with s_k ~ scale * N(0, 1); both
    (n, r) FP64, column-major, original point order."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, r)) / math.sqrt(n)
    s = scale * rng.standard_normal(r)
    return np.asfortranarray(U), np.asfortranarray(U * s[None, :])


def paper_problem(name: str, n: int = 262144) -> Workload:
    """A Sec. V-A kernel problem at n points: tol 1e-6, leaf 64, eta 0.7; the
    black-box sampler is an H2 matrix of the same kernel prebuilt at
    ``extra["operand_tol"]`` (ten times tighter than the target)."""
    if name == "exp3d":
        return Workload("exp3d", n, 3, K_EXP, (0.2, 0.0), tol=1e-6, sketch="h2matvec",
                        point_seed=6, omega_seed=43, extra={"operand_tol": 1e-7})
    if name == "helmholtz":
        return Workload("helmholtz", n, 3, K_HELMHOLTZ_IE, (3.0, 0.0), tol=1e-6,
                        sketch="h2matvec", point_seed=7, omega_seed=53,
                        extra={"operand_tol": 1e-7})
    if name == "update":
        # the covariance H2 of exp3d plus a symmetric rank-32 product whose
        # weights are of the order of the matrix's largest entries times n
        return Workload("update", n, 3, K_H2SUM, (), tol=1e-6, sketch="h2sum",
                        point_seed=6, omega_seed=63,
                        extra={"operands": [(K_EXP, (0.2, 0.0))], "operand_tol": 1e-7,
                               "rank": 32, "lowrank_seed": 64, "lowrank_scale": 0.01 * n})
    raise KeyError(name)
