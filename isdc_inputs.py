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

    def as_dict(self):
        return asdict(self)

    @property
    def N(self):
        return self.n ** self.ndim


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
