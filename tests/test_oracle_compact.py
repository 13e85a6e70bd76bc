"""Pins for the oracle's 4th-order compact discretisation (Sec. 3, Eq. 5): the
9-point Laplacian L_9 and the weighting matrix W, their multigrid, the exact
sine-transform solves, and the W-form SDC sweep with its W^{-1} residual.

The dense forms come from Kronecker products of the 1D second difference
(L_9 = D_xx + D_yy + (h^2/6) D_xx D_yy, W = I + (h^2/12) L_5), a construction
independent of the oracle's stencil loops."""
import numpy as np
import pytest

import oracle as O
import dense_ops as D
from isdc_inputs import initial_condition, sine_mode

C = O.STENCIL_COMPACT


def test_compact_operators_match_kronecker_forms():
    n, a, om = 7, 0.013, 0.7
    rng = np.random.default_rng(1)
    u, b = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    L9, W = D.laplacian9(n), D.weighting(n)
    np.testing.assert_allclose(O.laplacian9(u).reshape(-1), L9 @ u.reshape(-1), rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(O.apply_w(u).reshape(-1), W @ u.reshape(-1), rtol=0, atol=1e-14)
    H = W - a * L9
    r = b.reshape(-1) - H @ u.reshape(-1)
    np.testing.assert_allclose(O.residual9(a, u, b).reshape(-1), r, rtol=0, atol=1e-12)
    xj = u.reshape(-1) + om * r / np.diag(H)
    np.testing.assert_allclose(O.smooth_jacobi9(a, om, u, b).reshape(-1), xj, rtol=0, atol=1e-12)


@pytest.mark.parametrize("a", [0.0, 0.002, 0.3])
def test_compact_exact_and_dense_solves(a):
    n = 7
    b = np.random.default_rng(2).standard_normal((n, n))
    H = D.weighting(n) - a * D.laplacian9(n)
    x = np.linalg.solve(H, b.reshape(-1))
    np.testing.assert_allclose(O.solve_exact9(a, b).reshape(-1), x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.dense_solve9(a, b).reshape(-1), x, rtol=0, atol=1e-13)


def test_compact_stencil_is_fourth_order_and_five_point_second():
    """On sin(pi x) sin(pi y) the semi-discrete rate W^{-1} L_9 approaches the
    continuous -2 pi^2 with O(h^4) error (factor ~16 per halving of h); the
    5-point rate with O(h^2) (factor ~4)."""
    def rates(n):
        v = sine_mode(2, n)
        p = (n // 2, n // 2)
        lam9 = (O.laplacian9(v)[p] / v[p]) / (O.apply_w(v)[p] / v[p])
        lam5 = O.laplacian(v)[p] / v[p]
        return abs(lam9 + 2 * np.pi ** 2), abs(lam5 + 2 * np.pi ** 2)
    e9a, e5a = rates(15)
    e9b, e5b = rates(31)
    assert 14.0 < e9a / e9b < 17.0, e9a / e9b
    assert 3.8 < e5a / e5b < 4.2, e5a / e5b


def test_compact_multigrid_converges_to_exact_solve():
    n, a = 63, 0.001
    p = O.Problem(2, n, 1.0, 3, 0.01, stencil=C, smoother=O.SMOOTHER_JACOBI, nu1=1, nu2=1)
    b = np.random.default_rng(3).standard_normal((n, n))
    xe = O.solve_exact9(a, b)
    x, errs = np.zeros((n, n)), []
    for _ in range(30):
        x = O.vcycle(p, a, x, b)
        errs.append(np.abs(x - xe).max())
    assert errs[-1] < 1e-12 * np.abs(xe).max()
    rho = (errs[8] / errs[4]) ** 0.25
    assert 0.15 < rho < 0.40, rho   # measured 0.30 (damped Jacobi V(1,1), omega = 2/3)


def _compact_collocation(p: O.Problem, u0):
    """U = 1 (x) u0 + dt (Q (x) I) F(U), F(U_j) = W^{-1} nu L_9 U_j + f^E(U_j),
    solved directly (Newton + dense LU for u - u^3)."""
    N, M = p.N, p.M
    Q = O.q_matrix(M, p.nodes)
    A = np.linalg.solve(D.weighting(p.n), p.nu * D.laplacian9(p.n))
    u0v = u0.reshape(-1)
    if p.reaction == O.REACTION_NONE:
        U = np.linalg.solve(np.eye(M * N) - p.dt * np.kron(Q, A), np.tile(u0v, M))
        return U.reshape((M,) + p.shape)
    U = np.tile(u0v, M)
    for _ in range(50):
        Us = U.reshape(M, N)
        F = Us @ A.T + Us - Us ** 3
        G = U - np.tile(u0v, M) - p.dt * (np.kron(Q, np.eye(N)) @ F.reshape(-1))
        J = np.eye(M * N) - p.dt * np.kron(Q, np.eye(N)) @ np.block(
            [[(A + np.diag(1 - 3 * Us[j] ** 2)) if i == j else np.zeros((N, N)) for j in range(M)]
             for i in range(M)])
        dU = np.linalg.solve(J, G)
        U -= dU
        if np.abs(dU).max() < 1e-15:
            break
    return U.reshape((M,) + p.shape)


@pytest.mark.parametrize("kind", [O.NODES_LOBATTO, O.NODES_RADAU_RIGHT, O.NODES_LEGENDRE])
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_compact_sweeps_reproduce_collocation_solution(kind, solver):
    p = O.Problem(2, 7, 0.5, 3, 0.02, reaction=O.REACTION_ALLEN_CAHN, stencil=C, smoother=O.SMOOTHER_JACOBI,
                  solver=solver, tol=1e-14, max_sweeps=200, nodes=kind)
    u0 = initial_condition(2, 7, seed=14, noise_std=0.05)
    ref = _compact_collocation(p, u0)
    r = O.isdc_step(p, u0, 0, 2, want_nodes=True)
    assert r.status == 0
    np.testing.assert_allclose(r.nodes, ref, rtol=0, atol=1e-12)
    if kind == O.NODES_LEGENDRE:
        A = np.linalg.solve(D.weighting(7), 0.5 * D.laplacian9(7))
        w = O.end_weights(3, kind)
        F = [A @ ref[j].reshape(-1) + (ref[j] - ref[j] ** 3).reshape(-1) for j in range(3)]
        end = u0 + p.dt * sum(w[j] * F[j] for j in range(3)).reshape(p.shape)
    else:
        end = ref[-1]
    np.testing.assert_allclose(r.u, end, rtol=0, atol=1e-12)
    assert O.sdc_residual(p, r.nodes, u0) < 1e-13


@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_compact_sine_mode_decays_by_pade_factor(solver):
    """Pure diffusion on a sine mode: the rate is z = dt nu lambda_9 / lambda_W and
    converged SDC (Lobatto IIIA, M = 3) multiplies by R(z) = (1 + z/2 + z^2/12)/(1 - z/2 + z^2/12)."""
    from golden_io import pade_numerators
    n, nu, dt = 15, 1.0, 0.002
    v = sine_mode(2, n, (2, 1, 1))
    c = (n // 2, n // 2 + 1)
    z = dt * nu * (O.laplacian9(v)[c] / v[c]) / (O.apply_w(v)[c] / v[c])
    num = np.array(pade_numerators()[3])
    R = np.polyval(num[::-1], z) / np.polyval(num[::-1], -z)
    p = O.Problem(2, n, nu, 3, dt, reaction=O.REACTION_NONE, stencil=C, solver=solver, tol=1e-15, max_sweeps=300)
    u = v.copy()
    for _ in range(3):
        u = O.isdc_step(p, u, 0, 2).u
    np.testing.assert_allclose(u, R ** 3 * v, rtol=0, atol=1e-13)


def test_compact_heat_step_converges_fourth_order_in_space():
    """The heat equation of Sec. 4.1 with u_0 = sin(pi x) sin(pi y): with time
    error negligible (M = 5, tiny dt), the error against exp(-2 pi^2 nu t) u_0
    falls ~16x per halving of h with the compact stencil (~4x with 5 points)."""
    def err(n, stencil):
        p = O.Problem(2, n, 1.0, 5, 0.001, reaction=O.REACTION_NONE, stencil=stencil, solver=O.SOLVER_EXACT,
                      tol=1e-15, max_sweeps=100)
        u0 = sine_mode(2, n)
        u = u0.copy()
        for _ in range(5):
            u = O.isdc_step(p, u, 0, 0).u
        return np.abs(u - np.exp(-2 * np.pi ** 2 * 0.005) * u0).max()
    assert 13.0 < err(15, C) / err(31, C) < 18.0
    assert 3.5 < err(15, O.STENCIL_SECOND_ORDER) / err(31, O.STENCIL_SECOND_ORDER) < 4.5


def test_compact_residual_of_nodes_and_invalid_combinations():
    p = O.Problem(2, 15, 0.2, 3, 0.02, stencil=C, smoother=O.SMOOTHER_JACOBI)
    u0 = initial_condition(2, 15, seed=15)
    r = O.isdc_step(p, u0, 3, 2, want_nodes=True)
    assert abs(O.sdc_residual(p, r.nodes) - r.residuals[-1]) <= 1e-15 * max(1.0, r.residuals[-1])
    with pytest.raises(ValueError):
        O.isdc_step(O.Problem(3, 7, 0.2, 3, 0.02, stencil=C), initial_condition(3, 7, seed=1), 1, 2)
    with pytest.raises(ValueError):
        O.isdc_step(O.Problem(2, 7, 0.2, 3, 0.02, stencil=C, smoother=O.SMOOTHER_RBGS),
                    initial_condition(2, 7, seed=1), 1, 2)
