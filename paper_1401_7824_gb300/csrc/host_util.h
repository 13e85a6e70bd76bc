// host_util.h -- host-side tables shared by the single-instance context and
// the batched engine: collocation tables (Sec. 2, Eq. 2: Gauss-Lobatto,
// Gauss-Radau and Gauss-Legendre nodes, Q, full-step weights) and the dense
// inverse of the side-3 multigrid operator.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace isdc {
namespace host {

// ---------------------------------------------------------------------------
// Collocation tables (Sec. 2, Eq. 2).
// ---------------------------------------------------------------------------

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal alpha and squared off-diagonals beta (Sturm sequence count).
inline int sturm_count(const std::vector<double>& alpha, const std::vector<double>& beta, int size, double x) {
  int count = 0;
  double q = alpha[0] - x;  // leading principal minor ratio
  if (q < 0) ++count;
  for (int k = 1; k < size; ++k) {
    const double prev = (q == 0.0) ? 1e-300 : q;
    q = alpha[k] - x - beta[k - 1] / prev;
    if (q < 0) ++count;
  }
  return count;
}

// Eigenvalues (ascending) of that matrix, all inside (-1, 1), by bisection on
// the Sturm count: the Golub-Welsch nodes of the orthogonal polynomial whose
// recurrence coefficients alpha, beta are given.
inline void jacobi_matrix_eigs(const std::vector<double>& alpha, const std::vector<double>& beta, int size,
                               double* out) {
  for (int e = 0; e < size; ++e) {  // e-th smallest eigenvalue
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (sturm_count(alpha, beta, size, mid) > e) hi = mid; else lo = mid;
    }
    out[e] = 0.5 * (lo + hi);
  }
}

// Gauss-Lobatto nodes on [0,1].  The interior nodes are the roots of
// P'_{M-1}, i.e. of the Jacobi polynomial P^{(1,1)}_{M-2}: eigenvalues of its
// Jacobi matrix (zero diagonal, squared off-diagonals k(k+2)/((2k+1)(2k+3))).
inline void lobatto_nodes(int M, double* tau) {
  const int size = M - 2;
  std::vector<double> alpha(std::max(size, 1), 0.0), beta(std::max(size, 1)), x(std::max(size, 1));
  for (int k = 1; k < size; ++k) beta[k - 1] = double(k) * (k + 2) / ((2.0 * k + 1) * (2.0 * k + 3));
  jacobi_matrix_eigs(alpha, beta, size, x.data());
  tau[0] = 0.0;
  tau[M - 1] = 1.0;
  for (int e = 0; e < size; ++e) tau[e + 1] = 0.5 * (x[e] + 1.0);
}

// Right Gauss-Radau nodes on [0,1] (tau_M = 1).  The other M-1 nodes are the
// roots of the Jacobi polynomial P^{(1,0)}_{M-1} (weight 1 - x on [-1,1]):
// diagonal -1/((2k+1)(2k+3)), squared off-diagonals k(k+1)/(2k+1)^2.
inline void radau_right_nodes(int M, double* tau) {
  const int size = M - 1;
  std::vector<double> alpha(size), beta(size), x(size);
  for (int k = 0; k < size; ++k) alpha[k] = -1.0 / ((2.0 * k + 1) * (2.0 * k + 3));
  for (int k = 1; k < size; ++k) beta[k - 1] = double(k) * (k + 1) / ((2.0 * k + 1) * (2.0 * k + 1));
  jacobi_matrix_eigs(alpha, beta, size, x.data());
  for (int e = 0; e < size; ++e) tau[e] = 0.5 * (x[e] + 1.0);
  tau[M - 1] = 1.0;
}

// Gauss-Legendre nodes on [0,1]: roots of P_M, eigenvalues of the Legendre
// Jacobi matrix (zero diagonal, squared off-diagonals k^2/(4k^2-1)).
inline void legendre_nodes(int M, double* tau) {
  std::vector<double> alpha(M, 0.0), beta(M), x(M);
  for (int k = 1; k < M; ++k) beta[k - 1] = double(k) * k / (4.0 * k * k - 1.0);
  jacobi_matrix_eigs(alpha, beta, M, x.data());
  for (int e = 0; e < M; ++e) tau[e] = 0.5 * (x[e] + 1.0);
}

// Node family kind: 0 Gauss-Lobatto, 1 Gauss-Radau (right), 2 Gauss-Legendre.
inline void collocation_nodes(int kind, int M, double* tau) {
  if (kind == 1) radau_right_nodes(M, tau);
  else if (kind == 2) legendre_nodes(M, tau);
  else lobatto_nodes(M, tau);
}

// Integrals of the Lagrange basis over the nodes tau from 0 to each of the
// points t[0..npts-1]: out[p*M + j] = int_0^{t_p} l_j(s) ds, computed exactly
// (l_j expanded in powers of x = 2s - 1 in [-1,1], integrated term by term).
inline void lagrange_integrals(int M, const double* tau, int npts, const double* t, double* out) {
  std::vector<double> x(M);
  for (int i = 0; i < M; ++i) x[i] = 2.0 * tau[i] - 1.0;
  for (int j = 0; j < M; ++j) {
    std::vector<double> c(1, 1.0);  // coefficients, ascending powers
    double denom = 1.0;
    for (int i = 0; i < M; ++i) {
      if (i == j) continue;
      std::vector<double> nc(c.size() + 1, 0.0);
      for (size_t k = 0; k < c.size(); ++k) {
        nc[k + 1] += c[k];
        nc[k] -= x[i] * c[k];
      }
      c.swap(nc);
      denom *= (x[j] - x[i]);
    }
    auto antider = [&](double v) {
      double acc = 0.0, pw = v;
      for (size_t k = 0; k < c.size(); ++k) {
        acc += c[k] * pw / double(k + 1);
        pw *= v;
      }
      return acc;
    };
    const double base = antider(-1.0);
    for (int p = 0; p < npts; ++p) out[p * M + j] = 0.5 * (antider(2.0 * t[p] - 1.0) - base) / denom;
  }
}

// Q[m][j] = int_0^{tau_m} l_j(s) ds.
inline void q_matrix(int M, const double* tau, double* Q) { lagrange_integrals(M, tau, M, tau, Q); }

// Full-step weights w_j = int_0^1 l_j(s) ds.
inline void end_weights(int M, const double* tau, double* w) {
  const double one = 1.0;
  lagrange_integrals(M, tau, 1, &one, w);
}

// Inverse of the dense matrix of H = I - a L_h on a side-3 grid (Gauss-Jordan
// with partial pivoting), row-major, Np x Np.
inline void coarse_inverse(int dim, double a, std::vector<double>& inv) {
  const int n = 3, Np = dim == 2 ? 9 : 27;
  const double h = 1.0 / (n + 1), c = a / (h * h), d = 1.0 + 2.0 * dim * c;
  std::vector<double> A(Np * Np, 0.0);
  for (int p = 0; p < Np; ++p) {
    const int i = p % n, j = (p / n) % n, k = dim == 3 ? p / (n * n) : 0;
    A[p * Np + p] = d;
    const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    for (int q = 0; q < 2 * dim; ++q) {
      const int ii = nb[q][0], jj = nb[q][1], kk = nb[q][2];
      if (ii < 0 || ii >= n || jj < 0 || jj >= n || kk < 0 || kk >= (dim == 3 ? n : 1)) continue;
      A[p * Np + (ii + n * (jj + n * kk))] = -c;
    }
  }
  inv.assign(Np * Np, 0.0);
  for (int p = 0; p < Np; ++p) inv[p * Np + p] = 1.0;
  for (int col = 0; col < Np; ++col) {
    int piv = col;
    for (int r = col + 1; r < Np; ++r)
      if (std::fabs(A[r * Np + col]) > std::fabs(A[piv * Np + col])) piv = r;
    if (piv != col)
      for (int q = 0; q < Np; ++q) {
        std::swap(A[col * Np + q], A[piv * Np + q]);
        std::swap(inv[col * Np + q], inv[piv * Np + q]);
      }
    const double s = 1.0 / A[col * Np + col];
    for (int q = 0; q < Np; ++q) { A[col * Np + q] *= s; inv[col * Np + q] *= s; }
    for (int r = 0; r < Np; ++r) {
      if (r == col) continue;
      const double f = A[r * Np + col];
      if (f == 0.0) continue;
      for (int q = 0; q < Np; ++q) { A[r * Np + q] -= f * A[col * Np + q]; inv[r * Np + q] -= f * inv[col * Np + q]; }
    }
  }
}

// Inverse of the dense 9 x 9 matrix of W - a L_9 (4th-order compact stencil,
// 2D) on the side-3 grid, row-major.
inline void coarse_inverse9(double a, std::vector<double>& inv) {
  const int n = 3, Np = 9;
  const double h = 1.0 / (n + 1), q = a / (6.0 * h * h);
  const double c0 = 8.0 / 12.0 + 20.0 * q, ce = 1.0 / 12.0 - 4.0 * q, cc = -q;
  std::vector<double> A(Np * Np, 0.0);
  for (int p = 0; p < Np; ++p) {
    const int i = p % n, j = p / n;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
        const int nz = (di != 0) + (dj != 0);
        A[p * Np + ii + n * jj] = nz == 0 ? c0 : (nz == 1 ? ce : cc);
      }
  }
  inv.assign(Np * Np, 0.0);
  for (int p = 0; p < Np; ++p) inv[p * Np + p] = 1.0;
  for (int col = 0; col < Np; ++col) {
    int piv = col;
    for (int r = col + 1; r < Np; ++r)
      if (std::fabs(A[r * Np + col]) > std::fabs(A[piv * Np + col])) piv = r;
    if (piv != col)
      for (int c = 0; c < Np; ++c) {
        std::swap(A[col * Np + c], A[piv * Np + c]);
        std::swap(inv[col * Np + c], inv[piv * Np + c]);
      }
    const double s = 1.0 / A[col * Np + col];
    for (int c = 0; c < Np; ++c) { A[col * Np + c] *= s; inv[col * Np + c] *= s; }
    for (int r = 0; r < Np; ++r) {
      if (r == col) continue;
      const double f = A[r * Np + col];
      if (f == 0.0) continue;
      for (int c = 0; c < Np; ++c) { A[r * Np + c] -= f * A[col * Np + c]; inv[r * Np + c] -= f * inv[col * Np + c]; }
    }
  }
}

// Inverse of the dense matrix of I - a L_h on the periodic side-4 grid
// (h = 1/2; 16 or 64 unknowns, x fastest), row-major.
inline void coarse_inverse_per(int dim, double a, std::vector<double>& inv) {
  const int n = 4, Np = dim == 2 ? 16 : 64;
  const double h = 0.5, c = a / (h * h), d = 1.0 + 2.0 * dim * c;
  std::vector<double> A(size_t(Np) * Np, 0.0);
  for (int p = 0; p < Np; ++p) {
    const int i = p % n, j = (p / n) % n, k = dim == 3 ? p / (n * n) : 0;
    A[size_t(p) * Np + p] = d;
    const int nb[6][3] = {{(i + 3) % n, j, k}, {(i + 1) % n, j, k}, {i, (j + 3) % n, k},
                          {i, (j + 1) % n, k}, {i, j, (k + 3) % n}, {i, j, (k + 1) % n}};
    for (int q = 0; q < 2 * dim; ++q)
      A[size_t(p) * Np + (nb[q][0] + n * (nb[q][1] + n * nb[q][2]))] -= c;
  }
  inv.assign(size_t(Np) * Np, 0.0);
  for (int p = 0; p < Np; ++p) inv[size_t(p) * Np + p] = 1.0;
  for (int col = 0; col < Np; ++col) {
    int piv = col;
    for (int r = col + 1; r < Np; ++r)
      if (std::fabs(A[size_t(r) * Np + col]) > std::fabs(A[size_t(piv) * Np + col])) piv = r;
    if (piv != col)
      for (int q = 0; q < Np; ++q) {
        std::swap(A[size_t(col) * Np + q], A[size_t(piv) * Np + q]);
        std::swap(inv[size_t(col) * Np + q], inv[size_t(piv) * Np + q]);
      }
    const double sc = 1.0 / A[size_t(col) * Np + col];
    for (int q = 0; q < Np; ++q) { A[size_t(col) * Np + q] *= sc; inv[size_t(col) * Np + q] *= sc; }
    for (int r = 0; r < Np; ++r) {
      if (r == col) continue;
      const double f = A[size_t(r) * Np + col];
      if (f == 0.0) continue;
      for (int q = 0; q < Np; ++q) {
        A[size_t(r) * Np + q] -= f * A[size_t(col) * Np + q];
        inv[size_t(r) * Np + q] -= f * inv[size_t(col) * Np + q];
      }
    }
  }
}

// Rewrite the kernel-to-kernel edges of a captured graph as programmatic
// dependencies on the upstream kernel's launch-completion port: a downstream
// kernel may be launched once every block of the upstream one has started, and
// its blocks wait at entry (grid_dep_wait) until the upstream kernel has
// completed and its writes are visible.  Launch processing of each kernel then
// overlaps the kernel before it; the order of all memory effects is unchanged.
// Edges that touch non-kernel nodes (copies, memsets, events) stay ordinary.
inline cudaError_t programmatic_edges(cudaGraph_t g) {
  size_t ne = 0;
  cudaError_t e = cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne);
  if (e != cudaSuccess || ne == 0) return e;
  std::vector<cudaGraphNode_t> from(ne), to(ne);
  std::vector<cudaGraphEdgeData> data(ne);
  if ((e = cudaGraphGetEdges(g, from.data(), to.data(), data.data(), &ne)) != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> f, t;
  for (size_t q = 0; q < ne; ++q) {
    cudaGraphNodeType a, b;
    if (cudaGraphNodeGetType(from[q], &a) != cudaSuccess || cudaGraphNodeGetType(to[q], &b) != cudaSuccess) continue;
    if (a == cudaGraphNodeTypeKernel && b == cudaGraphNodeTypeKernel && data[q].type == cudaGraphDependencyTypeDefault &&
        data[q].from_port == cudaGraphKernelNodePortDefault) {
      f.push_back(from[q]);
      t.push_back(to[q]);
    }
  }
  if (f.empty()) return cudaSuccess;
  std::vector<cudaGraphEdgeData> plain(f.size()), prog(f.size());
  std::memset(plain.data(), 0, plain.size() * sizeof(cudaGraphEdgeData));
  std::memset(prog.data(), 0, prog.size() * sizeof(cudaGraphEdgeData));
  for (auto& d : prog) {
    d.from_port = cudaGraphKernelNodePortLaunchCompletion;
    d.type = cudaGraphDependencyTypeProgrammatic;
  }
  if ((e = cudaGraphRemoveDependencies(g, f.data(), t.data(), plain.data(), f.size())) != cudaSuccess) return e;
  return cudaGraphAddDependencies(g, f.data(), t.data(), prog.data(), f.size());
}

}  // namespace host
}  // namespace isdc
