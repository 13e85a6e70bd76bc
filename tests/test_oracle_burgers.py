"""Pins for the oracle's viscous Burgers equation of Sec. 4.1: periodic grid,
periodic multigrid, the exact solve by the discrete Fourier transform, the
5th-order WENO advection (Jiang-Shu, local Lax-Friedrichs splitting), and the
IMEX sweep on it.  Each pin is something the mathematics fixes independently of
the oracle's loops: Kronecker forms, exactness on quadratics, the ENO choice at
a jump, conservation, the convergence order on smooth data, translation
invariance, and the directly solved collocation system."""
import numpy as np
import pytest

import oracle as O
import dense_ops as D

B = O.EQUATION_BURGERS


def grid(n):
    h = 2.0 / n
    x = -1.0 + h * np.arange(n)
    return np.meshgrid(x, x, indexing="xy")


def gaussian(n, sigma=0.1):
    X, Y = grid(n)
    return np.exp(-(X ** 2 + Y ** 2) / sigma ** 2)


@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_periodic_operators_match_kronecker_forms(d, n):
    rng = np.random.default_rng(20 + d)
    u, b = rng.standard_normal((n,) * d), rng.standard_normal((n,) * d)
    L = D.laplacian_periodic(d, n)
    np.testing.assert_allclose(O.laplacian_per(u).reshape(-1), L @ u.reshape(-1), rtol=1e-13, atol=1e-11)
    a, om = 0.003, 0.7
    H = np.eye(n ** d) - a * L
    r = b.reshape(-1) - H @ u.reshape(-1)
    np.testing.assert_allclose(O.residual_per(a, u, b).reshape(-1), r, rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.smooth_jacobi_per(a, om, u, b).reshape(-1), u.reshape(-1) + om * r / np.diag(H),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.solve_exact_per(a, b).reshape(-1), np.linalg.solve(H, b.reshape(-1)),
                               rtol=0, atol=1e-12)


def test_periodic_transfers_are_adjoint():
    """Full weighting is 2^-d times the transpose of linear interpolation."""
    n, nc = 16, 8
    P = np.zeros((n * n, nc * nc))
    for c in range(nc * nc):
        e = np.zeros(nc * nc)
        e[c] = 1.0
        P[:, c] = O.prolong_per(e.reshape(nc, nc), np.zeros((n, n))).reshape(-1)
    R = np.zeros((nc * nc, n * n))
    for f in range(n * n):
        e = np.zeros(n * n)
        e[f] = 1.0
        R[:, f] = O.restrict_per(e.reshape(n, n)).reshape(-1)
    np.testing.assert_allclose(R, P.T / 4.0, rtol=0, atol=1e-15)
    assert np.allclose(P.sum(axis=1), 1.0)  # interpolation reproduces constants


@pytest.mark.parametrize("smoother,nu1", [(O.SMOOTHER_JACOBI, 1), (O.SMOOTHER_RBGS, 2)])
def test_periodic_multigrid_converges_to_exact_solve(smoother, nu1):
    n, a = 64, 0.002
    p = O.Problem(2, n, 1.0, 3, 0.01, equation=B, smoother=smoother, nu1=nu1, nu2=nu1)
    b = np.random.default_rng(4).standard_normal((n, n))
    xe = O.solve_exact_per(a, b)
    x, errs = np.zeros((n, n)), []
    for _ in range(40):
        x = O.vcycle(p, a, x, b)
        errs.append(np.abs(x - xe).max())
    assert errs[-1] < 1e-12 * np.abs(xe).max()
    rho = (errs[6] / errs[2]) ** 0.25
    # measured 0.39 (damped Jacobi V(1,1)) and 0.06 (red-black V(2,2))
    assert rho < (0.45 if smoother == O.SMOOTHER_JACOBI else 0.15), rho


def test_weno5_is_exact_on_quadratics_and_picks_the_smooth_stencil():
    """Finite-difference WENO reconstructs the flux h from point values that are
    cell averages of h; every 3-point candidate is exact for quadratic h, so the
    face value is exact whatever the weights.  At a jump the weights of the
    stencils crossing it vanish (ENO property)."""
    rng = np.random.default_rng(5)
    dx = 0.1
    for _ in range(5):
        c = rng.standard_normal(3)
        H = lambda x: c[0] * x + c[1] * x ** 2 / 2 + c[2] * x ** 3 / 3   # antiderivative of h
        h = lambda x: c[0] + c[1] * x + c[2] * x ** 2
        xs = dx * np.arange(-2, 3)
        avg = (H(xs + dx / 2) - H(xs - dx / 2)) / dx
        assert abs(O.weno5_face(avg) - h(dx / 2)) < 1e-13
    assert abs(O.weno5_face(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))) < 1e-9
    assert abs(O.weno5_face(np.array([0.0, 0.0, 1.0, 1.0, 1.0])) - 1.0) < 1e-9


def test_burgers_advection_conserves_and_converges_fifth_order():
    """Conservative differences of a periodic flux sum to zero; on smooth data the
    error against -(u u_x + u u_y) falls by about 2^5 per halving of h."""
    def err(n):
        X, Y = grid(n)
        u = 1.5 + np.sin(np.pi * X) * np.sin(np.pi * Y)
        fe = O.burgers_advection(u)
        assert abs(fe.sum()) < 1e-9 * np.abs(fe).sum()
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        return np.abs(fe + u * (ux + uy)).max()
    e = [err(n) for n in (32, 64, 128)]
    assert np.log2(e[1] / e[2]) > 4.5, e


def test_burgers_step_is_translation_invariant_and_conserves_mass():
    """Every operator of the step is shift invariant on the periodic grid, so
    stepping a shifted field gives the shifted result (to rounding: the
    multigrid hierarchy and the dense coarsest solve order their sums
    differently); the Laplacian and the flux differences both sum to zero, so
    with exact node solves the mean is conserved."""
    n = 32
    u0 = gaussian(n, 0.3) + 0.01 * np.random.default_rng(6).standard_normal((n, n))
    p = O.Problem(2, n, 0.2, 3, 0.01, equation=B, smoother=O.SMOOTHER_RBGS, nu1=2, nu2=2)
    a = O.isdc_step(p, u0, 4, 2).u
    b = O.isdc_step(p, np.roll(u0, (3, 5), axis=(0, 1)), 4, 2).u
    np.testing.assert_allclose(b, np.roll(a, (3, 5), axis=(0, 1)), rtol=0, atol=1e-12)
    # with exact node solves (multigrid cycles need not keep the sum of each solve)
    pe = O.Problem(2, n, 0.2, 3, 0.01, equation=B, solver=O.SOLVER_EXACT)
    c = O.isdc_step(pe, u0, 4, 0).u
    assert abs(c.sum() - u0.sum()) < 1e-12 * np.abs(u0).sum()


def _burgers_collocation(p, u0):
    """U = 1 (x) u0 + dt (Q (x) I) F(U), F = nu L_per U + f^E(U), by Newton with a
    finite-difference Jacobian (f^E from the oracle: this pins the sweep, the
    multigrid and the quadrature, not WENO itself)."""
    N, M = p.N, p.M
    Q = O.q_matrix(M, p.nodes)
    L = p.nu * D.laplacian_periodic(p.ndim, p.n)
    u0v = u0.reshape(-1)
    def F(U):
        Us = U.reshape(M, N)
        return np.concatenate([L @ Us[j] + O.burgers_advection(Us[j].reshape(p.shape)).reshape(-1)
                               for j in range(M)])
    def G(U):
        return U - np.tile(u0v, M) - p.dt * (np.kron(Q, np.eye(N)) @ F(U))
    U = np.tile(u0v, M)
    for _ in range(30):
        g = G(U)
        J = np.empty((M * N, M * N))
        eps = 1e-7
        for c in range(M * N):
            e = np.zeros(M * N)
            e[c] = eps
            J[:, c] = (G(U + e) - G(U - e)) / (2 * eps)
        dU = np.linalg.solve(J, g)
        U -= dU
        if np.abs(dU).max() < 1e-14:
            break
    return U.reshape((M,) + p.shape)


@pytest.mark.parametrize("kind", [O.NODES_LOBATTO, O.NODES_RADAU_RIGHT])
@pytest.mark.parametrize("solver", [O.SOLVER_EXACT, O.SOLVER_ISDC])
def test_burgers_sweeps_reproduce_collocation_solution(kind, solver):
    n = 8
    u0 = gaussian(n, 0.4)
    p = O.Problem(2, n, 0.1, 3, 0.02, equation=B, smoother=O.SMOOTHER_JACOBI, solver=solver, tol=1e-14,
                  max_sweeps=200, nodes=kind)
    ref = _burgers_collocation(p, u0)
    r = O.isdc_step(p, u0, 0, 2, want_nodes=True)
    assert r.status == 0
    np.testing.assert_allclose(r.nodes, ref, rtol=0, atol=1e-11)
    assert O.sdc_residual(p, r.nodes, u0) < 1e-13


def test_burgers_invalid_grids():
    for n in (12, 4):
        with pytest.raises(ValueError):
            O.isdc_step(O.Problem(2, n, 0.1, 3, 0.01, equation=B), np.zeros((n, n)), 1, 2)


def test_weno5_weights_follow_the_smoothness_indicator_definition():
    """Jiang-Shu define the candidate p_k as the quadratic with the cell averages
    of its 3-cell stencil, its smoothness indicator as
    beta_k = sum_{l=1,2} dx^(2l-1) int_cell (p_k^(l))^2, and the weights as
    d_k/(eps + beta_k)^2 normalised, d = (1/10, 6/10, 3/10), eps = 1e-6.  The
    face value is sum_k w_k p_k(x_{i+1/2}); recomputed here from polynomials."""
    rng = np.random.default_rng(7)
    dx = 1.0
    centers = dx * np.arange(-2, 3)          # cells i-2..i+2, cell i centred at 0
    for _ in range(20):
        v = rng.standard_normal(5) * rng.choice([0.01, 1.0, 10.0])
        faces, betas = [], []
        for k in range(3):
            cells = centers[k:k + 3]
            # cell averages of a0 + a1 x + a2 x^2 over [c - dx/2, c + dx/2]
            A = np.array([[1.0, c, c * c + dx * dx / 12.0] for c in cells])
            a = np.linalg.solve(A, v[k:k + 3])
            p = np.polynomial.Polynomial(a)
            faces.append(p(dx / 2))
            beta = 0.0
            for l in (1, 2):
                dl = p.deriv(l)
                sq = (dl * dl).integ()
                beta += dx ** (2 * l - 1) * (sq(dx / 2) - sq(-dx / 2))
            betas.append(beta)
        w = np.array([0.1, 0.6, 0.3]) / (1e-6 + np.array(betas)) ** 2
        ref = float(np.dot(w / w.sum(), faces))
        assert abs(O.weno5_face(v) - ref) <= 1e-12 * max(1.0, abs(ref)), (v, ref)


@pytest.mark.parametrize("kind", [O.NODES_LOBATTO, O.NODES_RADAU_RIGHT])
def test_first_burgers_sweep_is_imex_euler(kind):
    """Sec. 4.1: IMEX Euler is the base method.  From the spread start u^0 = u_0
    the first sweep of Eq. 4 reduces to IMEX Euler sub-steps over the points
    t_0 <= t_1 < ...: (I - dt_m nu L) u_{m+1} = u_m + dt_m f^E(u_m)."""
    n, nu, dt, M = 16, 0.3, 0.02, 3
    u0 = gaussian(n, 0.35)
    p = O.Problem(2, n, nu, M, dt, equation=B, solver=O.SOLVER_EXACT, nodes=kind)
    r = O.isdc_step(p, u0, 1, 0, want_nodes=True)
    tau = O.nodes(M, kind)
    pts = tau if kind == O.NODES_LOBATTO else np.concatenate([[0.0], tau])
    L = nu * D.laplacian_periodic(2, n)
    u = u0.reshape(-1)
    ref = []
    for m in range(len(pts) - 1):
        dtm = dt * (pts[m + 1] - pts[m])
        u = np.linalg.solve(np.eye(n * n) - dtm * L, u + dtm * O.burgers_advection(u.reshape(n, n)).reshape(-1))
        ref.append(u.reshape(n, n))
    got = r.nodes[1:] if kind == O.NODES_LOBATTO else r.nodes
    np.testing.assert_allclose(got, np.array(ref), rtol=0, atol=1e-13)
