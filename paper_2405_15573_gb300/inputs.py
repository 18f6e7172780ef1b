"""Seeded synthetic inputs shared by the library's callers, the tests and the oracle.

This module only *generates data*: surface point clouds and right-hand-side vectors, plus the
parameter sets of the synthetic Helmholtz-on-surface workloads. It holds none of the method's
arithmetic (no kernel entries, trees, compression or products), so that the oracle and the CUDA
path can both take their inputs from here without sharing any computation.

The paper's experiments use Galerkin BEM meshes that are not available here (Section 6.1); the
workloads below are collocation operators on Fibonacci-lattice spheres and ellipsoids whose
wavenumber-times-spacing lies inside the paper's range of kappa*h (Table 2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def fibonacci_sphere(n: int) -> np.ndarray:
    """Points i = 0..n-1 of the Fibonacci lattice on the unit sphere, shape (n, 3), float64.

    z_i = 1 - (2i+1)/n, rho_i = sqrt(1 - z_i^2), theta_i = i * pi * (3 - sqrt(5)),
    p_i = (rho_i cos theta_i, rho_i sin theta_i, z_i).
    """
    if n <= 0:
        return np.zeros((0, 3))
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    theta = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(theta), rho * np.sin(theta), z], axis=1)


def ellipsoid_points(n: int, axes=(1.0, 1.0, 1.0), radial_noise: float = 0.0,
                     seed: int = 0) -> np.ndarray:
    """Fibonacci lattice mapped to the ellipsoid with semi-axes `axes`.

    Each point is scaled componentwise by the semi-axes; with `radial_noise` = a > 0 it is then
    multiplied by (1 + a*u_i), u_i uniform on [-1, 1] from numpy's PCG64 stream `seed`.
    """
    p = fibonacci_sphere(n) * np.asarray(axes, dtype=np.float64)[None, :]
    if radial_noise:
        u = np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)
        p = p * (1.0 + radial_noise * u)[:, None]
    return p


def complex_normal(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex standard normal vector (or n x nrhs matrix): (g1 + i g2)/sqrt(2), g ~ N(0,1).

    Drawn from numpy's PCG64 stream `seed`: first all real parts, then all imaginary parts,
    in column-major order of the (n, nrhs) result.
    """
    m = 1 if nrhs is None else nrhs
    g = np.random.default_rng(seed).standard_normal(size=(2, m, n))
    x = ((g[0] + 1j * g[1]) / math.sqrt(2.0)).T  # (n, m)
    x = np.ascontiguousarray(x) if nrhs is not None else x[:, 0].copy()
    return x


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic Helmholtz-on-surface operator and its construction parameters."""
    name: str
    n: int
    wavenumber: float
    leaf: int
    eta: float
    eps: float
    tol_aca: float
    axes: tuple = (1.0, 1.0, 1.0)
    radial_noise: float = 0.0
    geom_seed: int = 0
    x_seed: int = 0
    nrhs: int = 1

    def points(self) -> np.ndarray:
        if self.axes == (1.0, 1.0, 1.0) and not self.radial_noise:
            return fibonacci_sphere(self.n)
        return ellipsoid_points(self.n, self.axes, self.radial_noise, self.geom_seed)

    def x(self) -> np.ndarray:
        return complex_normal(self.n, self.x_seed, None if self.nrhs == 1 else self.nrhs)


# Parity case: unit sphere, N = 2048, k = 4, leaf 32, eta = 1, ACA 1e-8, eps 1e-6, complex128.
SPHERE_2048 = Workload("sphere-N2048-k4", 2048, 4.0, 32, 1.0, 1e-6, 1e-8)
# Headline case: unit sphere, N = 32768, k = 16, leaf 64, eta = 1, eps 1e-6 (ACA at eps/100).
SPHERE_32768 = Workload("sphere-N32768-k16", 32768, 16.0, 64, 1.0, 1e-6, 1e-8)
SPHERE_32768_R32 = dataclasses.replace(SPHERE_32768, name="sphere-N32768-k16-R32", nrhs=32)
# Large multi-RHS case: ellipsoid (1, 0.7, 0.4), 1% radial noise, N = 131072, k = 32, eps 1e-4.
ELLIPSOID_131072_R64 = Workload("ellipsoid-N131072-k32-R64", 131072, 32.0, 64, 1.0, 1e-4, 1e-6,
                                axes=(1.0, 0.7, 0.4), radial_noise=0.01, nrhs=64)


def batched_pool(count: int = 256, seed0: int = 0) -> list[Workload]:
    """Many independent small operators: N log-uniform in [1024, 16384], sphere or ellipsoid
    (axes uniform in [0.5, 1]), k uniform in [1, 16], leaf 32, eta 1, eps 1e-6; seeds seed0..
    """
    out = []
    for j in range(count):
        r = np.random.default_rng(seed0 + j)
        n = int(round(math.exp(r.uniform(math.log(1024), math.log(16384)))))
        k = float(r.uniform(1.0, 16.0))
        if r.uniform() < 0.5:
            axes = (1.0, 1.0, 1.0)
        else:
            axes = tuple(float(a) for a in r.uniform(0.5, 1.0, size=3))
        out.append(Workload(f"pool{j}-N{n}", n, k, 32, 1.0, 1e-6, 1e-8, axes=axes,
                            geom_seed=seed0 + j, x_seed=seed0 + j))
    return out


def serving_pool(count: int = 64, seed0: int = 1000, n_lo: int = 4096, n_hi: int = 65536) -> list[Workload]:
    """Resident operators of the serving workload: N uniform in [n_lo, n_hi], k uniform in
    [2, 24], sphere or ellipsoid (axes uniform in [0.5, 1]), leaf 32, eta 1, eps 1e-6 (ACA 1e-8);
    seeds seed0.."""
    out = []
    for j in range(count):
        r = np.random.default_rng(seed0 + j)
        n = int(r.integers(n_lo, n_hi + 1))
        k = float(r.uniform(2.0, 24.0))
        if r.uniform() < 0.5:
            axes = (1.0, 1.0, 1.0)
        else:
            axes = tuple(float(a) for a in r.uniform(0.5, 1.0, size=3))
        out.append(Workload(f"serve{j}-N{n}", n, k, 32, 1.0, 1e-6, 1e-8, axes=axes,
                            geom_seed=seed0 + j, x_seed=seed0 + j))
    return out


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of `count` requests of a Poisson process of the given rate."""
    return np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=count))
