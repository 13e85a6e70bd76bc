"""Accumulated V-cycles (sweeps) of classical SDC and ISDC on the heat equation
of Sec. 4.1, computed with the oracle, beside the paper's Table 1a.

TEST INFRASTRUCTURE: runs the oracle only.
Usage: python -m oracle.table1 [--compact | --burgers]

Settings: unit square, u0 = sin(pi x) sin(pi y), zero Dirichlet values, one
step dt = 0.001, 63^2 interior points (dx = 1/64), the 5-point Laplacian or,
with --compact, the paper's 4th-order compact stencil with the weighting
matrix W (Sec. 3, Eq. 5), SDC residual < 5e-8.  With --burgers, Table 1b: the
viscous Burgers equation of Sec. 4.1 on the periodic [-1,1)^2 with 128^2 points
(dx = 1/64), u0 = exp(-(x^2 + y^2)/sigma^2), sigma = 0.1, WENO5 advection,
nu in {0.1, 1, 10}, the same dt, tolerance and multigrid choices.  Classical SDC: V-cycles
until the node residual is <= mg_tol.  ISDC: at most L = 2 V-cycles per node
solve, stopping early at the same mg_tol (the paper's counts are below
K~(M-1)L, so L acts as a cap).  The paper does not describe its multigrid
solver or its tolerance; mg_tol = 5e-9 and damped-Jacobi V(3,3) are this
table's choices.
"""
from __future__ import annotations

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
from isdc_inputs import sine_mode  # noqa: E402

# Table 1b of the paper (viscous Burgers): (nu, M) -> (SDC cycles, SDC sweeps, ISDC cycles, ISDC sweeps)
PAPER_TABLE_1B = {
    (0.1, 3): (21, 8, 21, 8), (0.1, 5): (26, 6, 26, 6), (0.1, 7): (33, 5, 33, 5),
    (1, 3): (97, 17, 66, 17), (1, 5): (140, 17, 117, 17), (1, 7): (160, 15, 143, 15),
    (10, 3): (207, 25, 100, 25), (10, 5): (523, 38, 298, 38), (10, 7): (902, 50, 578, 50),
}

# Table 1a of the paper: (nu, M) -> (SDC cycles, SDC sweeps, ISDC cycles, ISDC sweeps)
PAPER_TABLE_1A = {
    (1, 3): (16, 4, 12, 4), (1, 5): (23, 3, 20, 3), (1, 7): (32, 3, 28, 3),
    (10, 3): (36, 5, 20, 5), (10, 5): (61, 5, 40, 5), (10, 7): (79, 4, 47, 4),
    (100, 3): (106, 13, 52, 13), (100, 5): (150, 10, 104, 13), (100, 7): (187, 9, 167, 14),
}


def heat_problem(nu, M, solver, smoother=O.SMOOTHER_JACOBI, nu1=3, nu2=3, mg_tol=5e-9,
                 stencil=O.STENCIL_SECOND_ORDER):
    return O.Problem(2, 63, float(nu), M, 0.001, reaction=O.REACTION_NONE, smoother=smoother, nu1=nu1, nu2=nu2,
                     solver=solver, tol=5e-8, max_sweeps=100, mg_tol=mg_tol, mg_max_cycles=100, stencil=stencil)


def burgers_problem(nu, M, solver, smoother=O.SMOOTHER_JACOBI, nu1=3, nu2=3, mg_tol=5e-9, n=128):
    return O.Problem(2, n, float(nu), M, 0.001, equation=O.EQUATION_BURGERS, smoother=smoother, nu1=nu1, nu2=nu2,
                     solver=solver, tol=5e-8, max_sweeps=100, mg_tol=mg_tol, mg_max_cycles=100)


def burgers_initial(n=128, sigma=0.1):
    """u0 = exp(-(x^2 + y^2)/sigma^2) on the periodic grid x_i = -1 + 2i/n (x fastest)."""
    import numpy as np
    x = -1.0 + (2.0 / n) * np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return np.exp(-(X ** 2 + Y ** 2) / sigma ** 2)


def table_burgers(n=128):
    u0 = burgers_initial(n)
    rows = {}
    for nu in (0.1, 1, 10):
        for M in (3, 5, 7):
            sdc = O.isdc_step(burgers_problem(nu, M, O.SOLVER_MG_TOL, n=n), u0, 0, 0)
            isdc = O.isdc_step(burgers_problem(nu, M, O.SOLVER_ISDC_CAPPED, n=n), u0, 0, 2)
            rows[(nu, M)] = (sdc.vcycles, sdc.sweeps, isdc.vcycles, isdc.sweeps)
    return rows


def table(smoother=O.SMOOTHER_JACOBI, nu1=3, nu2=3, mg_tol=5e-9, stencil=O.STENCIL_SECOND_ORDER):
    u0 = sine_mode(2, 63)
    rows = {}
    for nu in (1, 10, 100):
        for M in (3, 5, 7):
            sdc = O.isdc_step(heat_problem(nu, M, O.SOLVER_MG_TOL, smoother, nu1, nu2, mg_tol, stencil), u0, 0, 0)
            isdc = O.isdc_step(heat_problem(nu, M, O.SOLVER_ISDC_CAPPED, smoother, nu1, nu2, mg_tol, stencil),
                               u0, 0, 2)
            rows[(nu, M)] = (sdc.vcycles, sdc.sweeps, isdc.vcycles, isdc.sweeps)
    return rows


def main():
    compact = "--compact" in sys.argv[1:]
    burgers = "--burgers" in sys.argv[1:]
    rows = table_burgers() if burgers else table(stencil=O.STENCIL_COMPACT if compact else O.STENCIL_SECOND_ORDER)
    paper = PAPER_TABLE_1B if burgers else PAPER_TABLE_1A
    print("| nu | M | SDC (this) | ISDC (this) | savings | SDC (paper) | ISDC (paper) | savings (paper) |")
    print("|---|---|---|---|---|---|---|---|")
    for (nu, M), (sc, ss, ic, isw) in rows.items():
        pc, ps, pic, pis = paper[(nu, M)]
        print(f"| {nu} | {M} | {sc}({ss}) | {ic}({isw}) | {100 * (1 - ic / sc):.0f} % | {pc}({ps}) | {pic}({pis}) "
              f"| {100 * (1 - pic / pc):.0f} % |")


if __name__ == "__main__":
    main()
