"""Dense-matrix forms of the 5/7-point operators, built from Kronecker products
of the 1D second-difference matrix (textbook construction, independent of the
oracle's stencil loops).  Used only on tiny grids to pin the oracle."""
import numpy as np


def lap1d(n):
    h = 1.0 / (n + 1)
    return (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2


def laplacian(d, n):
    """L_h on interior points, C order with x fastest (index i + n*j [+ n^2*k])."""
    L1, I = lap1d(n), np.eye(n)
    if d == 2:
        return np.kron(I, L1) + np.kron(L1, I)
    return (np.kron(I, np.kron(I, L1)) + np.kron(I, np.kron(L1, I)) + np.kron(L1, np.kron(I, I)))


def helmholtz(d, n, a):
    """I - a L_h"""
    return np.eye(n ** d) - a * laplacian(d, n)


def red_mask(d, n):
    """True where i+j(+k) is even with 1-based interior indices."""
    g = np.indices((n,) * d).sum(axis=0) + d  # 0-based indices sum + d
    return (g % 2 == 0).reshape(-1)


def laplacian9(n):
    """The 4th-order compact Laplacian as D_xx + D_yy + (h^2/6) D_xx D_yy
    (Kronecker products of the 1D second difference; 2D)."""
    h = 1.0 / (n + 1)
    L1, I = lap1d(n), np.eye(n)
    return np.kron(I, L1) + np.kron(L1, I) + h ** 2 / 6.0 * np.kron(L1, L1)


def weighting(n):
    """W = I + (h^2/12) L_5 (2D)."""
    h = 1.0 / (n + 1)
    return np.eye(n * n) + h ** 2 / 12.0 * laplacian(2, n)


def lap1d_periodic(n, h):
    """Circulant 1D second difference on n periodic points."""
    L = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    L[0, -1] = L[-1, 0] = 1.0
    return L / h ** 2


def laplacian_periodic(d, n):
    """Periodic L_h on [-1,1)^d with h = 2/n (Kronecker form, x fastest)."""
    L1, I = lap1d_periodic(n, 2.0 / n), np.eye(n)
    if d == 2:
        return np.kron(I, L1) + np.kron(L1, I)
    return np.kron(I, np.kron(I, L1)) + np.kron(I, np.kron(L1, I)) + np.kron(L1, np.kron(I, I))
