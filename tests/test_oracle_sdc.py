"""Pins for the oracle's SDC / ISDC time step (Sec. 2 Eq. 4, Sec. 3, Sec. 4).

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's code: the collocation solution solved
directly, the order gained per sweep, the Pade closed form on sine modes, the
collocation fixed point, and the paper's qualitative claims."""
import numpy as np
import pytest

import oracle as O
import dense_ops as D
from golden_io import pade_numerators
from isdc_inputs import initial_condition, sine_mode


def _collocation_solution(p: O.Problem, u0, reaction_fn=None):
    """Solve U = 1 (x) u0 + dt (Q (x) I) F(U) directly (the M*N collocation system
    whose solution converged SDC reproduces, Sec. 1-2).  F(U_j) = nu L U_j + f^E(U_j)."""
    N, M = p.N, p.M
    Q = O.q_matrix(M, p.nodes)
    A = p.nu * D.laplacian(p.ndim, p.n)
    u0v = u0.reshape(-1)
    if p.reaction in (O.REACTION_NONE, O.REACTION_LINEAR):
        Aj = A + (p.lambda_e * np.eye(N) if p.reaction == O.REACTION_LINEAR else 0.0)
        big = np.eye(M * N) - p.dt * np.kron(Q, Aj)
        U = np.linalg.solve(big, np.tile(u0v, M))
        return U.reshape((M,) + p.shape)
    # Allen-Cahn: Newton on G(U) = U - 1(x)u0 - dt (Q(x)I) F(U)
    U = np.tile(u0v, M)
    for _ in range(50):
        Us = U.reshape(M, N)
        F = (Us @ A.T) + Us - Us ** 3
        G = U - np.tile(u0v, M) - p.dt * (np.kron(Q, np.eye(N)) @ F.reshape(-1))
        J = np.eye(M * N) - p.dt * np.kron(Q, np.eye(N)) @ np.block(
            [[(A + np.diag(1 - 3 * Us[j] ** 2)) if i == j else np.zeros((N, N)) for j in range(M)]
             for i in range(M)])
        dU = np.linalg.solve(J, G)
        U -= dU
        if np.abs(dU).max() < 1e-15:
            break
    return U.reshape((M,) + p.shape)


CASES = [
    # ndim, n, nu, M, dt, reaction, smoother
    (2, 7, 1.0, 3, 0.01, O.REACTION_NONE, O.SMOOTHER_JACOBI),
    (2, 7, 0.5, 5, 0.02, O.REACTION_ALLEN_CAHN, O.SMOOTHER_JACOBI),
    (3, 3, 0.3, 5, 0.05, O.REACTION_ALLEN_CAHN, O.SMOOTHER_RBGS),
    (3, 7, 0.1, 3, 0.02, O.REACTION_ALLEN_CAHN, O.SMOOTHER_RBGS),
    (2, 7, 0.2, 7, 0.05, O.REACTION_LINEAR, O.SMOOTHER_RBGS),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_converged_sweeps_reproduce_collocation_solution(case, solver):
    d, n, nu, M, dt, reaction, smoother = case
    nu1 = 1 if smoother == O.SMOOTHER_JACOBI else 2
    p = O.Problem(d, n, nu, M, dt, reaction=reaction, lambda_e=-0.7, smoother=smoother,
                  nu1=nu1, nu2=nu1, solver=solver, tol=1e-14, max_sweeps=200)
    u0 = initial_condition(d, n, seed=11, noise_std=0.05)
    ref = _collocation_solution(p, u0)
    r = O.isdc_step(p, u0, 0, 2, want_nodes=True)
    assert r.status == 0
    np.testing.assert_allclose(r.nodes, ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.u, ref[-1], rtol=0, atol=1e-12)


@pytest.mark.parametrize("M,ks", [(3, [1, 2, 3, 4, 5]), (5, [1, 2, 3, 4])])
def test_order_increases_by_one_per_sweep(M, ks):
    """Dahlquist problem y' = (lambda_I + lambda_E) y (Sec. 1: each sweep raises
    the order by one up to the collocation order 2M-2).  A sine mode on the
    3x3 grid is an eigenvector of L_h, so the grid problem is exactly scalar."""
    n = 3
    h = 1.0 / (n + 1)
    lam_h = -8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    nu = 1.5 / -lam_h          # lambda_I = -1.5
    lam_e = 0.5                # lambda_E = +0.5 (explicit part)
    v = sine_mode(2, n)
    T = 1.0
    for k in ks:
        errs = []
        for steps in (4, 8, 16):
            p = O.Problem(2, n, nu, M, T / steps, reaction=O.REACTION_LINEAR, lambda_e=lam_e,
                          solver=O.SOLVER_EXACT)
            u = v.copy()
            for _ in range(steps):
                u = O.isdc_step(p, u, k, 0).u
            errs.append(np.abs(u - np.exp(-1.0 * T) * v).max())
        order = np.log2(errs[1] / errs[2])
        expect = min(k, 2 * M - 2)
        assert abs(order - expect) < 0.35, (k, errs, order)


@pytest.mark.parametrize("M", [3, 5])
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_sine_mode_decays_by_pade_factor(M, solver):
    """Pure diffusion (f^E = 0) on a sine mode: converged SDC is the Lobatto IIIA
    collocation step, whose stability function is the (M-1,M-1) Pade
    approximant, so u_n = R(dt nu lambda_h)^n u_0 exactly (up to rounding)."""
    d, n, nu, dt = 2, 15, 1.0, 0.002
    p_mode = (2, 1, 1)
    h = 1.0 / (n + 1)
    lam = -4.0 / h ** 2 * sum(np.sin(p_mode[a] * np.pi * h / 2) ** 2 for a in range(d))
    z = dt * nu * lam
    c = np.array(pade_numerators()[M])
    R = np.polyval(c[::-1], z) / np.polyval(c[::-1], -z)
    p = O.Problem(d, n, nu, M, dt, reaction=O.REACTION_NONE, solver=solver, tol=1e-15,
                  max_sweeps=300)
    u = sine_mode(d, n, p_mode)
    v = u.copy()
    for _ in range(3):
        r = O.isdc_step(p, u, 0, 2)
        u = r.u
    np.testing.assert_allclose(u, R ** 3 * v, rtol=0, atol=1e-13)
    # and the continuous solution exp(-5 pi^2 nu t) to the spatial error O(h^2)
    exact = np.exp(-5 * np.pi ** 2 * nu * 3 * dt) * v
    assert np.abs(u - exact).max() < 0.05 * np.abs(exact).max() * (h / (1 / 16)) ** 2


@pytest.mark.parametrize("vcycles", [1, 2])
def test_collocation_solution_is_a_fixed_point_of_isdc(vcycles):
    p = O.Problem(2, 15, 0.3, 5, 0.03, reaction=O.REACTION_ALLEN_CAHN, solver=O.SOLVER_EXACT,
                  tol=1e-14, max_sweeps=200)
    u0 = initial_condition(2, 15, seed=3)
    coll = O.isdc_step(p, u0, 0, 0, want_nodes=True).nodes
    pi = O.Problem(2, 15, 0.3, 5, 0.03, reaction=O.REACTION_ALLEN_CAHN, solver=O.SOLVER_ISDC)
    r = O.isdc_step(pi, u0, 1, vcycles, want_nodes=True, nodes_in=coll)
    assert np.abs(r.nodes - coll).max() < 1e-13
    assert r.residuals[0] < 1e-13


def _stiff_heat(n=31, solver=O.SOLVER_ISDC, guess=O.GUESS_PREVIOUS_SWEEP, max_sweeps=60):
    # heat equation of Sec. 4.1 (nu = 10, dt = 0.001 on the unit square)
    return O.Problem(2, n, 10.0, 3, 0.001, reaction=O.REACTION_NONE, solver=solver, guess=guess,
                     tol=5e-8, max_sweeps=max_sweeps)


def test_isdc_needs_at_least_as_many_sweeps_as_sdc():
    """K <= K~ (Sec. 3) and ISDC spends fewer V-cycles than classical SDC solving
    each node to a tolerance (Sec. 4.2, Table 1 trend)."""
    u0 = sine_mode(2, 31)
    sdc = O.isdc_step(_stiff_heat(solver=O.SOLVER_EXACT), u0, 0, 0)
    isdc = O.isdc_step(_stiff_heat(), u0, 0, 2)
    mgsdc = O.isdc_step(O.Problem(2, 31, 10.0, 3, 0.001, reaction=O.REACTION_NONE,
                                  solver=O.SOLVER_MG_TOL, mg_tol=1e-12, tol=5e-8), u0, 0, 0)
    assert sdc.status == isdc.status == mgsdc.status == 0
    assert isdc.sweeps >= sdc.sweeps
    assert isdc.vcycles == isdc.sweeps * (3 - 1) * 2
    assert isdc.vcycles < mgsdc.vcycles


def test_many_vcycles_reproduce_exact_solve_sweep_by_sweep():
    u0 = initial_condition(2, 31, seed=5)
    ex = O.isdc_step(_stiff_heat(solver=O.SOLVER_EXACT), u0, 6, 0)
    mg = O.isdc_step(_stiff_heat(), u0, 6, 30)
    np.testing.assert_allclose(mg.residuals, ex.residuals, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(mg.u, ex.u, rtol=0, atol=1e-13)


@pytest.mark.parametrize("guess", [O.GUESS_ZERO, O.GUESS_LEFT_NODE])
def test_isdc_fails_without_previous_sweep_guess(guess):
    """Sec. 4.3: with a zero initial guess, or u_m^{k+1}, ISDC does not converge,
    while classical SDC (exact solves) still does."""
    u0 = initial_condition(2, 31, seed=6)
    bad = O.isdc_step(_stiff_heat(guess=guess, max_sweeps=60), u0, 0, 2)
    good = O.isdc_step(_stiff_heat(), u0, 0, 2)
    sdc = O.isdc_step(_stiff_heat(solver=O.SOLVER_EXACT, guess=guess), u0, 0, 0)
    assert good.status == 0 and sdc.status == 0
    assert bad.status == 1 and bad.residuals[-1] > 1e3 * 5e-8


def test_nonfinite_input_reports_status():
    p = O.Problem(2, 7, 0.1, 3, 0.05)
    u0 = initial_condition(2, 7, seed=1)
    u0[3, 3] = np.nan
    assert O.isdc_step(p, u0, 0, 2).status == 2


def test_workload_2d_127_isdc_matches_exact_solve_sdc():
    """The 127^2 workload: ISDC with 2 V(1,1) cycles against classical SDC with
    exact solves, both swept to residual 1e-10 for 10 steps; both approximate
    the same collocation solution."""
    from isdc_inputs import workload_2d_127
    w = workload_2d_127()
    u0 = initial_condition(2, w.n, w.seed)
    pi = O.Problem(2, w.n, w.nu, w.M, w.dt, smoother=O.SMOOTHER_JACOBI, max_sweeps=100)
    pe = O.Problem(2, w.n, w.nu, w.M, w.dt, solver=O.SOLVER_EXACT, max_sweeps=100)
    a = O.integrate(pi, u0, 3, 0, 2)
    b = O.integrate(pe, u0, 3, 0, 0)
    assert all(s == 0 for s in a.status + b.status)
    assert all(ka >= kb for ka, kb in zip(a.sweeps, b.sweeps))
    rel = np.linalg.norm(a.u - b.u) / np.linalg.norm(b.u)
    assert rel < 1e-9, rel


def test_sdc_residual_of_nodes_matches_step_history():
    p = O.Problem(2, 15, 0.2, 5, 0.02, reaction=O.REACTION_ALLEN_CAHN)
    u0 = initial_condition(2, 15, seed=9)
    r = O.isdc_step(p, u0, 3, 2, want_nodes=True)
    assert abs(O.sdc_residual(p, r.nodes) - r.residuals[-1]) <= 1e-15 * max(1.0, r.residuals[-1])
    # zero at the collocation solution, and equal to max|U_m - u_0| when f = 0
    coll = _collocation_solution(p, u0)
    assert O.sdc_residual(p, coll) < 1e-13
    p0 = O.Problem(2, 15, 1e-300, 5, 0.02, reaction=O.REACTION_NONE)
    nodes = np.stack([u0] + [u0 + 0.1 * m for m in range(1, 5)])
    assert abs(O.sdc_residual(p0, nodes) - 0.4) < 1e-12


# --- Gauss-Radau (right) and Gauss-Legendre nodes (Sec. 2) ----------------------
def _full_step_weights(tau):
    """w with sum_j w_j tau_j^p = 1/(p+1), p < M: the interpolatory rule on the
    nodes, from a Vandermonde solve (independent of the oracle's quadrature)."""
    M = len(tau)
    V = np.vander(tau, M, increasing=True).T
    return np.linalg.solve(V, 1.0 / np.arange(1, M + 1))


def _collocation_end(p, u0, U):
    """End value of the collocation step: the last node when tau_M = 1, else
    u0 + dt sum_j w_j f(U_j) (Gauss-Legendre)."""
    if p.nodes != O.NODES_LEGENDRE:
        return U[-1]
    A = p.nu * D.laplacian(p.ndim, p.n)
    w = _full_step_weights(O.nodes(p.M, p.nodes))
    F = [A @ U[j].reshape(-1) + (U[j] - U[j] ** 3).reshape(-1) if p.reaction == O.REACTION_ALLEN_CAHN
         else A @ U[j].reshape(-1) + (p.lambda_e * U[j].reshape(-1) if p.reaction == O.REACTION_LINEAR else 0.0)
         for j in range(p.M)]
    return u0 + p.dt * sum(w[j] * F[j] for j in range(p.M)).reshape(p.shape)


NODE_CASES = [
    # ndim, n, nu, M, dt, reaction, smoother, nodes
    (2, 7, 1.0, 3, 0.01, O.REACTION_NONE, O.SMOOTHER_JACOBI, O.NODES_RADAU_RIGHT),
    (2, 7, 0.5, 2, 0.02, O.REACTION_ALLEN_CAHN, O.SMOOTHER_RBGS, O.NODES_RADAU_RIGHT),
    (3, 3, 0.3, 5, 0.05, O.REACTION_ALLEN_CAHN, O.SMOOTHER_RBGS, O.NODES_LEGENDRE),
    (2, 7, 0.2, 3, 0.05, O.REACTION_LINEAR, O.SMOOTHER_JACOBI, O.NODES_LEGENDRE),
]


@pytest.mark.parametrize("case", NODE_CASES)
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_radau_legendre_sweeps_reproduce_collocation_solution(case, solver):
    d, n, nu, M, dt, reaction, smoother, kind = case
    nu1 = 1 if smoother == O.SMOOTHER_JACOBI else 2
    p = O.Problem(d, n, nu, M, dt, reaction=reaction, lambda_e=-0.7, smoother=smoother, nu1=nu1, nu2=nu1,
                  solver=solver, tol=1e-14, max_sweeps=200, nodes=kind)
    u0 = initial_condition(d, n, seed=12, noise_std=0.05)
    ref = _collocation_solution(p, u0)
    r = O.isdc_step(p, u0, 0, 2, want_nodes=True)
    assert r.status == 0
    np.testing.assert_allclose(r.nodes, ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.u, _collocation_end(p, u0, ref), rtol=0, atol=1e-12)
    assert O.sdc_residual(p, r.nodes, u0) < 1e-13
    # M node solves per sweep (t_0 is not a node)
    if solver == O.SOLVER_ISDC:
        assert r.vcycles == r.sweeps * M * 2


@pytest.mark.parametrize("kind,M,ks,conv", [(O.NODES_RADAU_RIGHT, 3, [1, 2, 3, 4], 5),
                                            (O.NODES_LEGENDRE, 2, [1, 2, 3], 4),
                                            (O.NODES_LEGENDRE, 3, [1, 2, 3, 4], 6)])
def test_radau_legendre_order_per_sweep(kind, M, ks, conv):
    """Dahlquist problem as above: each sweep gains one order at the nodes, up
    to the collocation order (2M-1 Radau IIA, 2M Gauss).  The Gauss step ends
    with the full-step quadrature of f at the nodes, one order above them."""
    n = 3
    h = 1.0 / (n + 1)
    lam_h = -8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    nu, lam_e, T = 1.5 / -lam_h, 0.5, 1.0
    v = sine_mode(2, n)
    for k in ks + [40]:
        errs = []
        for steps in (4, 8, 16):
            p = O.Problem(2, n, nu, M, T / steps, reaction=O.REACTION_LINEAR, lambda_e=lam_e,
                          solver=O.SOLVER_EXACT, nodes=kind)
            u = v.copy()
            for _ in range(steps):
                u = O.isdc_step(p, u, k, 0).u
            errs.append(np.abs(u - np.exp(-1.0 * T) * v).max())
        order = np.log2(errs[1] / errs[2])
        expect = min(k + (1 if kind == O.NODES_LEGENDRE else 0), conv)
        assert abs(order - expect) < 0.35, (k, errs, order)


@pytest.mark.parametrize("fam,kind,M", [("radau", O.NODES_RADAU_RIGHT, 2), ("radau", O.NODES_RADAU_RIGHT, 3),
                                        ("legendre", O.NODES_LEGENDRE, 2), ("legendre", O.NODES_LEGENDRE, 3)])
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_sine_mode_decays_by_radau_gauss_pade_factor(fam, kind, M, solver):
    """Pure diffusion on a sine mode: converged SDC is the Radau IIA / Gauss
    collocation step, whose stability function is the (M-1, M) / (M, M) Pade
    approximant of exp."""
    from golden_io import pade_radau_gauss
    d, n, nu, dt = 2, 15, 1.0, 0.002
    p_mode = (2, 1, 1)
    h = 1.0 / (n + 1)
    lam = -4.0 / h ** 2 * sum(np.sin(p_mode[a] * np.pi * h / 2) ** 2 for a in range(d))
    z = dt * nu * lam
    num, den = pade_radau_gauss()[(fam, M)]
    R = np.polyval(num[::-1], z) / np.polyval(den[::-1], z)
    p = O.Problem(d, n, nu, M, dt, reaction=O.REACTION_NONE, solver=solver, tol=1e-15, max_sweeps=300,
                  nodes=kind)
    u = sine_mode(d, n, p_mode)
    v = u.copy()
    for _ in range(3):
        u = O.isdc_step(p, u, 0, 2).u
    np.testing.assert_allclose(u, R ** 3 * v, rtol=0, atol=1e-13)


def test_radau_legendre_resume_and_residual_need_u0():
    p = O.Problem(2, 15, 0.2, 3, 0.02, nodes=O.NODES_LEGENDRE)
    u0 = initial_condition(2, 15, seed=13)
    full = O.isdc_step(p, u0, 5, 2, want_nodes=True)
    part = O.isdc_step(p, u0, 3, 2, want_nodes=True)
    rest = O.isdc_step(p, u0, 2, 2, want_nodes=True, nodes_in=part.nodes)
    np.testing.assert_array_equal(rest.nodes, full.nodes)
    np.testing.assert_array_equal(rest.u, full.u)
    assert abs(O.sdc_residual(p, full.nodes, u0) - full.residuals[-1]) <= 1e-15
    with pytest.raises(ValueError):
        O.sdc_residual(p, full.nodes)
