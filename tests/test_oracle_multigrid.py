"""Pins for the oracle's spatial operator and multigrid components (the
implicit solve of Sec. 3; the multigrid design itself is textbook, the paper
does not describe its solver)."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import dense_ops as D
from isdc_inputs import sine_mode

RNG = np.random.default_rng(1234)


@pytest.mark.parametrize("d,n", [(2, 7), (3, 7), (2, 15)])
def test_laplacian_matches_kronecker_form(d, n):
    u = RNG.standard_normal((n,) * d)
    np.testing.assert_allclose(O.laplacian(u).reshape(-1), D.laplacian(d, n) @ u.reshape(-1),
                               rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("d,n,p", [(2, 15, (2, 3, 1)), (3, 15, (1, 4, 2))])
def test_sine_modes_are_eigenvectors(d, n, p):
    h = 1.0 / (n + 1)
    lam = -4.0 / h ** 2 * sum(np.sin(p[a] * np.pi * h / 2) ** 2 for a in range(d))
    v = sine_mode(d, n, p)
    np.testing.assert_allclose(O.laplacian(v), lam * v, rtol=0, atol=1e-10 * abs(lam))


@pytest.mark.parametrize("d,n", [(2, 7), (3, 7)])
def test_residual(d, n):
    a = 0.013
    x, b = RNG.standard_normal((2,) + (n,) * d)
    r = b.reshape(-1) - D.helmholtz(d, n, a) @ x.reshape(-1)
    np.testing.assert_allclose(O.residual(a, x, b).reshape(-1), r, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,n", [(2, 7), (3, 7)])
def test_jacobi_sweep_is_damped_jacobi(d, n):
    a, w = 0.02, 2.0 / 3.0
    x, b = RNG.standard_normal((2,) + (n,) * d)
    A = D.helmholtz(d, n, a)
    xv = x.reshape(-1)
    ref = xv + w * (b.reshape(-1) - A @ xv) / np.diag(A)
    np.testing.assert_allclose(O.smooth_jacobi(a, w, x, b).reshape(-1), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,n", [(2, 7), (3, 7), (2, 8 - 1)])
def test_rbgs_is_gauss_seidel_in_red_black_order(d, n):
    # Gauss-Seidel with the unknowns ordered red first, then black:
    # (D + L) x_new = b - U x_old in that ordering.
    a = 0.05
    x, b = RNG.standard_normal((2,) + (n,) * d)
    A = D.helmholtz(d, n, a)
    red = D.red_mask(d, n)
    perm = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
    Ap = A[np.ix_(perm, perm)]
    lower = np.tril(Ap)
    upper = Ap - lower
    xp = sla.solve_triangular(lower, b.reshape(-1)[perm] - upper @ x.reshape(-1)[perm], lower=True)
    ref = np.empty_like(xp)
    ref[perm] = xp
    got = O.smooth_rbgs(a, x, b).reshape(-1)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    # after the sweep every black row is satisfied exactly
    r = b.reshape(-1) - A @ got
    assert np.abs(r[~red]).max() < 1e-12


def _dense_prolongation(d, nc):
    n = 2 * nc + 1
    P = np.zeros((n ** d, nc ** d))
    for c in range(nc ** d):
        e = np.zeros(nc ** d)
        e[c] = 1.0
        P[:, c] = O.prolong_add(e.reshape((nc,) * d), np.zeros((n,) * d)).reshape(-1)
    return P


def _dense_restriction(d, n):
    nc = (n - 1) // 2
    R = np.zeros((nc ** d, n ** d))
    for c in range(n ** d):
        e = np.zeros(n ** d)
        e[c] = 1.0
        R[:, c] = O.restrict_fw(e.reshape((n,) * d)).reshape(-1)
    return R


@pytest.mark.parametrize("d,nc", [(2, 3), (3, 3), (2, 7)])
def test_prolongation_is_tensor_hat(d, nc):
    n = 2 * nc + 1
    P = _dense_prolongation(d, nc)
    hat1 = np.zeros((n, nc))
    for I in range(1, nc + 1):
        hat1[2 * I - 1, I - 1] = 1.0      # fine 2I (1-based) -> row 2I-1 (0-based)
        hat1[2 * I - 2, I - 1] = 0.5
        hat1[2 * I, I - 1] = 0.5
    ref = np.kron(hat1, hat1) if d == 2 else np.kron(hat1, np.kron(hat1, hat1))
    np.testing.assert_array_equal(P, ref)


@pytest.mark.parametrize("d,n", [(2, 7), (3, 7), (2, 15)])
def test_full_weighting_is_scaled_transpose_of_interpolation(d, n):
    R = _dense_restriction(d, n)
    P = _dense_prolongation(d, (n - 1) // 2)
    np.testing.assert_allclose(R, P.T / 2 ** d, rtol=0, atol=1e-16)


@pytest.mark.parametrize("d,n,a", [(2, 3, 0.1), (3, 3, 0.7), (2, 7, 0.01)])
def test_dense_coarse_solve(d, n, a):
    b = RNG.standard_normal((n,) * d)
    ref = np.linalg.solve(D.helmholtz(d, n, a), b.reshape(-1))
    np.testing.assert_allclose(O.dense_solve(a, b).reshape(-1), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,n,a", [(2, 15, 0.01), (3, 7, 0.3), (2, 31, 5.0)])
def test_exact_sine_transform_solve(d, n, a):
    b = RNG.standard_normal((n,) * d)
    ref = np.linalg.solve(D.helmholtz(d, n, a), b.reshape(-1))
    got = O.solve_exact(a, b).reshape(-1)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def _contraction(problem, a, cycles=8):
    b = RNG.standard_normal(problem.shape)
    xs = O.solve_exact(a, b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(cycles):
        x = O.vcycle(problem, a, x, b)
        errs.append(np.abs(x - xs).max())
    return errs, x, xs


def test_vcycle_converges_to_exact_solution_2d_jacobi():
    p = O.Problem(2, 63, 1.0, 3, 1.0, smoother=O.SMOOTHER_JACOBI, nu1=1, nu2=1)
    a = 10.0   # a/h^2 ~ 4e4: Poisson-dominated, the hardest case for the cycle
    errs, x, xs = _contraction(p, a, cycles=40)
    rho = (errs[-1] / errs[9]) ** (1.0 / 30)
    # damped Jacobi (omega=2/3) V(1,1) on the 5-point operator: smoothing factor
    # 2/3 per sweep, two-grid factor ~ (2/3)^2; asymptotic band
    assert 0.3 < rho < 0.55, rho
    assert np.abs(x - xs).max() < 1e-12 * np.abs(xs).max()


def test_vcycle_converges_to_exact_solution_3d_rbgs():
    p = O.Problem(3, 31, 1.0, 5, 1.0, smoother=O.SMOOTHER_RBGS, nu1=2, nu2=2)
    a = 10.0
    errs, x, xs = _contraction(p, a, cycles=14)
    rho = (errs[6] / errs[1]) ** (1.0 / 5)
    # red-black Gauss-Seidel V(2,2), 7-point operator, full weighting
    assert 0.03 < rho < 0.15, rho
    assert np.abs(x - xs).max() < 1e-12 * np.abs(xs).max()


def test_vcycle_is_exact_on_coarsest_grid():
    p = O.Problem(3, 3, 1.0, 5, 1.0, smoother=O.SMOOTHER_RBGS, nu1=2, nu2=2)
    b = RNG.standard_normal(p.shape)
    x = O.vcycle(p, 0.4, np.zeros_like(b), b)
    np.testing.assert_allclose(x, O.solve_exact(0.4, b), atol=1e-13)


def _dense_smooth(kind, A, x, b, d, n, omega=2.0 / 3.0):
    if kind == O.SMOOTHER_JACOBI:
        return x + omega * (b - A @ x) / np.diag(A)
    red = D.red_mask(d, n)
    perm = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
    Ap = A[np.ix_(perm, perm)]
    lower = np.tril(Ap)
    xp = sla.solve_triangular(lower, b[perm] - (Ap - lower) @ x[perm], lower=True)
    out = np.empty_like(xp)
    out[perm] = xp
    return out


def _dense_vcycle(kind, d, n, a, x, b, nu1, nu2):
    """Textbook V-cycle in dense matrices: smooth, restrict the residual with
    R = P^T / 2^d, recurse on the rediscretised operator I - a L_{2h} from a
    zero guess, solve exactly on the side-3 grid, interpolate and add, smooth."""
    A = D.helmholtz(d, n, a)
    if n == 3:
        return np.linalg.solve(A, b)
    for _ in range(nu1):
        x = _dense_smooth(kind, A, x, b, d, n)
    nc = (n - 1) // 2
    P = _dense_prolongation(d, nc)
    rc = (P.T / 2 ** d) @ (b - A @ x)
    ec = _dense_vcycle(kind, d, nc, a, np.zeros(nc ** d), rc, nu1, nu2)
    x = x + P @ ec
    for _ in range(nu2):
        x = _dense_smooth(kind, A, x, b, d, n)
    return x


@pytest.mark.parametrize("d,n,kind,nu1,nu2", [(2, 7, O.SMOOTHER_JACOBI, 1, 1),
                                                (2, 15, O.SMOOTHER_JACOBI, 1, 1),
                                                (3, 7, O.SMOOTHER_RBGS, 2, 2),
                                                (2, 15, O.SMOOTHER_RBGS, 2, 1)])
def test_vcycle_matches_dense_multigrid_cycle(d, n, kind, nu1, nu2):
    a = 0.37
    x, b = RNG.standard_normal((2,) + (n,) * d)
    p = O.Problem(d, n, 1.0, 3, 1.0, smoother=kind, nu1=nu1, nu2=nu2)
    ref = _dense_vcycle(kind, d, n, a, x.reshape(-1), b.reshape(-1), nu1, nu2)
    np.testing.assert_allclose(O.vcycle(p, a, x, b).reshape(-1), ref, rtol=0, atol=1e-12)
