"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.  This module holds the workload recipes only (grid sizes,
parameters, initial data, random draws); none of the method's arithmetic lives
here, and it imports neither the oracle nor the CUDA package.

Grid convention: interior points of the unit square/cube, side n = 2^j - 1,
h = 1/(n+1), x_i = i*h for i = 1..n; arrays are float64 in C order with shape
(n, n) or (n, n, n) indexed [k, j, i] (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np


def grid_coords(n: int) -> np.ndarray:
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def sine_mode(ndim: int, n: int, p=(1, 1, 1)) -> np.ndarray:
    """prod_axes sin(p_a pi x_a) on the interior grid."""
    x = grid_coords(n)
    f = [np.sin(p[a] * np.pi * x) for a in range(ndim)]
    if ndim == 2:
        return np.ascontiguousarray(f[1][:, None] * f[0][None, :])
    return np.ascontiguousarray(f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :])


def initial_condition(ndim: int, n: int, seed: int, noise_std: float = 0.01) -> np.ndarray:
    """sin(pi x) sin(pi y) [sin(pi z)] plus N(0, noise_std^2) noise on interior
    points (PCG64 stream of `seed`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = sine_mode(ndim, n)
    return np.ascontiguousarray(u + noise_std * rng.standard_normal(u.shape))


@dataclass
class Workload:
    """One single-instance ISDC integration."""
    name: str
    ndim: int
    n: int
    nu: float
    M: int
    dt: float
    steps: int
    n_vcycles: int          # L, V-cycles per node solve
    smoother: int           # 0 damped Jacobi, 1 red-black Gauss-Seidel
    nu1: int
    nu2: int
    omega: float = 2.0 / 3.0
    reaction: int = 1       # u - u^3
    tol: float = 1e-10
    vcycle_fp32: bool = False
    seed: int = 1
    nodes: int = 0          # 0 Gauss-Lobatto, 1 Gauss-Radau (right), 2 Gauss-Legendre
    stencil: int = 0        # 0 5/7-point, 1 4th-order compact with W (2D)
    equation: int = 0       # 0 reaction-diffusion (Dirichlet), 1 viscous Burgers (periodic, n = 2^j)

    def as_dict(self):
        return asdict(self)

    @property
    def N(self):
        return self.n ** self.ndim


def periodic_grid_coords(n: int) -> np.ndarray:
    """x_i = -1 + 2 i / n, i = 0..n-1: the periodic grid on [-1, 1)."""
    return -1.0 + (2.0 / n) * np.arange(n, dtype=np.float64)


def periodic_bump(ndim: int, n: int, seed: int, sigma: float = 0.1, noise_std: float = 0.01) -> np.ndarray:
    """exp(-|x|^2 / sigma^2) on the periodic grid plus seeded N(0, noise_std^2)
    noise (x fastest): the Burgers initial value of Sec. 4.1 (sigma = 0.1)."""
    x = periodic_grid_coords(n)
    g = np.meshgrid(*([x] * ndim), indexing="ij")[::-1]
    r2 = sum(c ** 2 for c in g)
    u = np.exp(-r2 / sigma ** 2)
    if noise_std:
        u = u + noise_std * np.random.default_rng(seed).standard_normal(u.shape)
    return np.ascontiguousarray(u)


def workload_initial(w: "Workload") -> np.ndarray:
    """The workload's initial value: periodic bump (Burgers) or sine product + noise."""
    if w.equation == 1:
        return periodic_bump(w.ndim, w.n, w.seed)
    return initial_condition(w.ndim, w.n, w.seed)


def _log_uniform(rng, lo, hi):
    return float(10.0 ** rng.uniform(np.log10(lo), np.log10(hi)))


# The workloads: the 2D 127^2 ISDC case, the 3D 255^3 FP64 case and the 3D
# 511^3 mixed-precision case (nu drawn log-uniformly in [0.01, 1] from seed 3).
def workload_2d_127() -> Workload:
    return Workload("2d_n127_M3_fp64", 2, 127, 0.1, 3, 0.05, 10, 2, 0, 1, 1, seed=1)


def workload_3d_255() -> Workload:
    return Workload("3d_n255_M5_fp64", 3, 255, 0.1, 5, 0.02, 20, 2, 1, 2, 2, seed=2)


def workload_3d_511_mixed() -> Workload:
    rng = np.random.Generator(np.random.PCG64(3))
    nu = _log_uniform(rng, 0.01, 1.0)
    return Workload("3d_n511_M5_mixed", 3, 511, nu, 5, 0.02, 10, 2, 1, 2, 2,
                    vcycle_fp32=True, seed=3)


def batch_instances(count: int = 256, seed: int = 4, j_range=(6, 10)):
    """Independent 2D instances: side 2^j - 1 with j uniform in j_range,
    nu log-uniform in [0.01, 1], dt uniform in [0.01, 0.1], M in {3, 5}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        j = int(rng.integers(j_range[0], j_range[1] + 1))
        nu = _log_uniform(rng, 0.01, 1.0)
        dt = float(rng.uniform(0.01, 0.1))
        M = int(rng.choice([3, 5]))
        out.append(Workload(f"batch{b}", 2, 2 ** j - 1, nu, M, dt, 10, 2, 0, 1, 1,
                            vcycle_fp32=True, seed=seed * 100003 + b))
    return out


def batch_instances_3d(count: int = 32, seed: int = 6, j_range=(6, 8)):
    """Independent 3D instances (the 3D share of the request mix): side
    2^j - 1 with j uniform in j_range, nu log-uniform in [0.01, 1], dt uniform
    in [0.01, 0.1], M in {3, 5}; red-black Gauss-Seidel V(2,2) settings."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        j = int(rng.integers(j_range[0], j_range[1] + 1))
        nu = _log_uniform(rng, 0.01, 1.0)
        dt = float(rng.uniform(0.01, 0.1))
        M = int(rng.choice([3, 5]))
        out.append(Workload(f"batch3d{b}", 3, 2 ** j - 1, nu, M, dt, 10, 2, 1, 2, 2,
                            vcycle_fp32=True, seed=seed * 100003 + b))
    return out


def request_stream(count: int = 2000, rate: float = 200.0, seed: int = 5):
    """Poisson arrivals at `rate` per second; 70 % 2D (side 127..1023), 30 % 3D
    (side 63..255); M in {3, 5}; nu, dt drawn as for the batch; 10 steps each.
    Returns (arrival_time_s, Workload) pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate))
        if rng.uniform() < 0.7:
            ndim, j = 2, int(rng.integers(7, 11))
        else:
            ndim, j = 3, int(rng.integers(6, 9))
        nu = _log_uniform(rng, 0.01, 1.0)
        dt = float(rng.uniform(0.01, 0.1))
        M = int(rng.choice([3, 5]))
        sm, nu1, nu2 = (0, 1, 1) if ndim == 2 else (1, 2, 2)
        out.append((t, Workload(f"req{r}", ndim, 2 ** j - 1, nu, M, dt, 10, 2, sm, nu1, nu2,
                                vcycle_fp32=True, seed=seed * 100003 + r)))
    return out


def workload_3d_255_radau() -> Workload:
    """The 3D 255^3 FP64 workload with M = 5 right Gauss-Radau nodes (5 node solves per sweep)."""
    return Workload("3d_n255_M5_radau_fp64", 3, 255, 0.1, 5, 0.02, 20, 2, 1, 2, 2, seed=2, nodes=1)


def workload_3d_255_legendre() -> Workload:
    """The 3D 255^3 FP64 workload with M = 5 Gauss-Legendre nodes (end-point quadrature)."""
    return Workload("3d_n255_M5_legendre_fp64", 3, 255, 0.1, 5, 0.02, 20, 2, 1, 2, 2, seed=2, nodes=2)


def workload_2d_1023_compact() -> Workload:
    """2D heat-type problem with the 4th-order compact stencil and W (Sec. 3, Eq. 5):
    1023^2, nu = 0.1, dt = 0.01, M = 5, damped Jacobi V(2,2), L = 2."""
    return Workload("2d_n1023_M5_compact_fp64", 2, 1023, 0.1, 5, 0.01, 10, 2, 0, 2, 2, seed=6, stencil=1)


def workload_2d_1024_burgers() -> Workload:
    """Viscous Burgers of Sec. 4.1 on the periodic [-1,1)^2, 1024^2 points, nu = 0.1,
    dt = 0.0005, M = 5, red-black V(2,2), L = 2 (seeded noise on the Gaussian)."""
    return Workload("2d_n1024_M5_burgers_fp64", 2, 1024, 0.1, 5, 0.0005, 10, 2, 1, 2, 2, reaction=0, seed=7,
                    equation=1)
