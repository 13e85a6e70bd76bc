// compact_kernels.cuh -- sm_103a kernels of the 4th-order compact
// discretisation of Sec. 3 (Eq. 5), 2D.
//
//   L_9 u = (4 * edge neighbours + corner neighbours - 20 u) / (6 h^2)
//   W u   = (8 u + edge neighbours) / 12          (= u + (h^2/12) L_5 u)
//   W u' = nu L_9 u + W f^E(u),  f~ = W f^E + nu L_9 u
//
// Node solves: (W - a L_9) x = b with a = dt_m nu, i.e. c0 x + ce E(x) + cc C(x)
// = b with c0 = 2/3 + 10a/(3h^2), ce = 1/12 - 2a/(3h^2), cc = -a/(6h^2)
// (E, C: sums of the 4 edge / 4 corner neighbours).  The multigrid kernels work
// on the row-scaled form x - ke E(x) - kc C(x) = beta, ke = -ce/c0,
// kc = -cc/c0, beta = b/c0.  The 9-point operator couples points of the same
// red-black colour, so the smoother is damped Jacobi.
#pragma once
#include "sdc_kernels.cuh"

namespace isdc {

// Sum of the 4 corner (diagonal) neighbours of (i,j); zero outside the interior.
template <typename T>
__device__ __forceinline__ T corner_sum(const T* __restrict__ x, int i, int j, int n, int p) {
  const bool l = i > 0, r = i < n - 1, d = j > 0, u = j < n - 1;
  const T lo = (l && d ? x[p - n - 1] : T(0)) + (r && d ? x[p - n + 1] : T(0));
  const T hi = (l && u ? x[p + n - 1] : T(0)) + (r && u ? x[p + n + 1] : T(0));
  return lo + hi;
}

// ---------------------------------------------------------------------------
// Multigrid on (W - a L_9) x = b.
// ---------------------------------------------------------------------------
// Damped Jacobi: xo = x + omega (beta - x + ke E + kc C); zero_guess: x == 0.
template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_jacobi9(int n, T ke, T kc, T omega, const T* __restrict__ x, const T* __restrict__ beta, T* __restrict__ xo,
              int zero_guess) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  if (zero_guess) {
    xo[p] = omega * beta[p];
    return;
  }
  const T xp = x[p];
  const T r = fma(ke, nbsum<T, 2>(x, i, j, 0, n, p), fma(kc, corner_sum<T>(x, i, j, n, p), beta[p])) - xp;
  xo[p] = fma(omega, r, xp);
}

// Scaled residual r' = beta - x + ke E + kc C = (b - (W - a L_9) x) / c0.
template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_residual9(int n, T ke, T kc, const T* __restrict__ x, const T* __restrict__ beta, T* __restrict__ r) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  r[p] = fma(ke, nbsum<T, 2>(x, i, j, 0, n, p), fma(kc, corner_sum<T>(x, i, j, n, p), beta[p])) - x[p];
}

// Max-norm of the unscaled residual c0 * r' (classical SDC stopping test), FP64.
__global__ void __launch_bounds__(kBX* kBY)
    k_resnorm9(int n, double ke, double kc, double c0, const double* __restrict__ x, const double* __restrict__ beta,
               unsigned long long* __restrict__ out) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = i + n * j;
    const double r =
        c0 * (fma(ke, nbsum<double, 2>(x, i, j, 0, n, p), fma(kc, corner_sum<double>(x, i, j, n, p), beta[p])) - x[p]);
    rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
  }
  block_max_atomic(rb, out);
}

// Bottom of the compact V-cycle: every level with side <= the threshold in one
// block, in shared memory (local levels 0..nlev-1; the last is the side-3 grid
// solved with the precomputed c0 (W - a L_9)^{-1}).  Damped Jacobi, full
// weighting, bilinear interpolation: the grid-wide kernels' arithmetic.
struct BottomParams9 {
  int nlev;
  int side[kMaxLevels];
  double ke[kMaxLevels], kc[kMaxLevels];  // row-scaled edge / corner couplings per level
  double rscale[kMaxLevels];              // restriction factor c0_l / (16 c0_{l+1})
  int nu1, nu2;
  double omega;
  const double* G;  // c0 (W - a L_9)^{-1} on the side-3 grid, row-major 9 x 9
};

__device__ void bt9_smooth(const BottomParams9& P, int l, double* x, const double* b, double* t) {
  const int n = P.side[l], Np = n * n;
  for (int p = threadIdx.x; p < Np; p += blockDim.x) t[p] = x[p];
  __syncthreads();
  for (int p = threadIdx.x; p < Np; p += blockDim.x) {
    const int i = p % n, j = p / n;
    const double r =
        fma(P.ke[l], nbsum<double, 2>(t, i, j, 0, n, p), fma(P.kc[l], corner_sum<double>(t, i, j, n, p), b[p])) - t[p];
    x[p] = fma(P.omega, r, t[p]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBottomThreads)
    k_bottom9(BottomParams9 P, const double* __restrict__ b_top, double* __restrict__ x_top, int load_x) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* base = reinterpret_cast<double*>(smem_raw);
  double *X[kMaxLevels], *B[kMaxLevels], *Tt[kMaxLevels];
  int off = 0;
  for (int l = 0; l < P.nlev; ++l) {
    const int Np = P.side[l] * P.side[l];
    X[l] = base + off; off += Np;
    B[l] = base + off; off += Np;
    Tt[l] = base + off; off += Np;
  }
  {
    const int Np = P.side[0] * P.side[0];
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      B[0][p] = b_top[p];
      X[0][p] = load_x ? x_top[p] : 0.0;  // zero when entered as a coarse-grid correction
    }
  }
  __syncthreads();
  const int last = P.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const int n = P.side[l], nc = P.side[l + 1];
    for (int s = 0; s < P.nu1; ++s) bt9_smooth(P, l, X[l], B[l], Tt[l]);
    for (int p = threadIdx.x; p < n * n; p += blockDim.x) {
      const int i = p % n, j = p / n;
      Tt[l][p] = fma(P.ke[l], nbsum<double, 2>(X[l], i, j, 0, n, p),
                     fma(P.kc[l], corner_sum<double>(X[l], i, j, n, p), B[l][p])) - X[l][p];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
      B[l + 1][q] = restrict_point<double, 2, false>(nc, P.rscale[l], Tt[l], q % nc, q / nc, 0);
      X[l + 1][q] = 0.0;
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < 9; r += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < 9; ++q) acc = fma(P.G[r * 9 + q], B[last][q], acc);
    X[last][r] = acc;
  }
  __syncthreads();
  for (int l = last - 1; l >= 0; --l) {
    const int nc = P.side[l + 1];
    for (int q = threadIdx.x; q < (nc + 1) * (nc + 1); q += blockDim.x)
      prolong_cell<double, 2, false>(nc, X[l + 1], X[l], q % (nc + 1), q / (nc + 1), 0);
    __syncthreads();
    for (int s = 0; s < P.nu2; ++s) bt9_smooth(P, l, X[l], B[l], Tt[l]);
  }
  {
    const int Np = P.side[0] * P.side[0];
    for (int p = threadIdx.x; p < Np; p += blockDim.x) x_top[p] = X[0][p];
  }
}

// ---------------------------------------------------------------------------
// SDC sweep with the weighting matrix (Eq. 5), FP64.  Per point p the context
// stores U_p, Ft_p = f~(u_p) = W f^E(u_p) + nu L_9 u_p and G_p = nu L_9 u_p.
// ---------------------------------------------------------------------------
// f~ and nu L_9 u at one point (nu6 = nu / (6 h^2)).
__device__ __forceinline__ void ftilde_at(const double* __restrict__ u, int i, int j, int n, int p, double nu6,
                                          int reaction, double& ft, double& g) {
  const double up = u[p];
  g = nu6 * fma(4.0, nbsum<double, 2>(u, i, j, 0, n, p), fma(-20.0, up, corner_sum<double>(u, i, j, n, p)));
  double we = 0.0;
  if (reaction) {  // W f^E(u) = (8 f^E(u_p) + edge neighbours' f^E) / 12
    const bool l = i > 0, r = i < n - 1, d = j > 0, t = j < n - 1;
    const double e = (l ? reaction_term(reaction, u[p - 1]) : 0.0) + (r ? reaction_term(reaction, u[p + 1]) : 0.0) +
                     ((d ? reaction_term(reaction, u[p - n]) : 0.0) + (t ? reaction_term(reaction, u[p + n]) : 0.0));
    we = fma(8.0, reaction_term(reaction, up), e) * (1.0 / 12.0);
  }
  ft = we + g;
}

// Start of a step: every point u_p = u, Ft_p = f~(u), G_p = nu L_9 u.
__global__ void __launch_bounds__(kBX* kBY)
    k_spread9(int n, size_t N, double nu6, int reaction, int P, const double* __restrict__ u, double* __restrict__ U,
              double* __restrict__ Ft, double* __restrict__ G) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  double ft, g;
  ftilde_at(u, i, j, n, p, nu6, reaction, ft, g);
  const double up = u[p];
  for (int m = 0; m < P; ++m) {
    U[m * N + p] = up;
    Ft[m * N + p] = ft;
    G[m * N + p] = g;
  }
}

// Ft and G of one point's values (resume from given node values).
__global__ void __launch_bounds__(kBX* kBY)
    k_eval_f9(int n, double nu6, int reaction, const double* __restrict__ u, double* __restrict__ ft,
              double* __restrict__ g) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  double a, b;
  ftilde_at(u, i, j, n, p, nu6, reaction, a, b);
  ft[p] = a;
  g[p] = b;
}

// Right-hand side of Eq. 5 for the step from point m, row-scaled:
//   b = W (u_m^{k+1} + dt_m f^E(u_m^{k+1})) + C_m,
//   C_m = dt sum_j s_{m,j} f~_j^k - dt_m W f^E(u_m^k) - dt_m nu L_9 u_{m+1}^k,
// beta = b / c0.  For m >= 1 the same pass stores Ft_m and G_m of u_m^{k+1}.
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs9(int n, double nu6, int reaction, double dtm, double inv_c0, const double* __restrict__ Um,
           const double* __restrict__ Cm, double* __restrict__ beta, double* __restrict__ Ftm,
           double* __restrict__ Gm) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  auto v = [&](int q) {
    const double uq = Um[q];
    return fma(dtm, reaction_term(reaction, uq), uq);
  };
  const bool l = i > 0, r = i < n - 1, d = j > 0, t = j < n - 1;
  const double e = ((l ? v(p - 1) : 0.0) + (r ? v(p + 1) : 0.0)) + ((d ? v(p - n) : 0.0) + (t ? v(p + n) : 0.0));
  const double wv = fma(8.0, v(p), e) * (1.0 / 12.0);
  beta[p] = (wv + Cm[p]) * inv_c0;
  if (Ftm) {
    double ft, g;
    ftilde_at(Um, i, j, n, p, nu6, reaction, ft, g);
    Ftm[p] = ft;
    Gm[p] = g;
  }
}

// End of a sweep: Ft and G at the last point; for every point m >= 1 the
// W-weighted SDC residual
//   rho_m = W (u_0 - u_m) + dt sum_j q_{m,j} f~_j      (W r_m = rho_m, Sec. 3)
// into Rho[m-1]; and the next sweep's C_m.  Node j is point j + OFF.
template <int OFF, int P>
__global__ void __launch_bounds__(kBX* kBY)
    k_sweep_end9(int n, size_t N, double nu6, int reaction, SweepTables tb, const double* __restrict__ U,
                 double* __restrict__ Ft, double* __restrict__ G, double* __restrict__ C, double* __restrict__ Rho) {
  grid_dep_wait();
  constexpr int M = P - OFF;
  static_assert(M >= 2 && M <= kMaxM && P <= kMaxP, "point count out of range");
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  double ft[P], g[P], qf[P];
  const double* ul = U + (size_t)(P - 1) * N;
  ftilde_at(ul, i, j, n, p, nu6, reaction, ft[P - 1], g[P - 1]);
  Ft[(size_t)(P - 1) * N + p] = ft[P - 1];
  G[(size_t)(P - 1) * N + p] = g[P - 1];
#pragma unroll
  for (int m = 0; m < P - 1; ++m) {
    ft[m] = Ft[m * N + p];
    g[m] = G[m * N + p];
  }
  qf[0] = 0.0;
#pragma unroll
  for (int m = 1; m < P; ++m) {
    double acc = tb.dtQ[m][0] * ft[OFF];
#pragma unroll
    for (int jj = 1; jj < M; ++jj) acc = fma(tb.dtQ[m][jj], ft[jj + OFF], acc);
    qf[m] = acc;
  }
  // W (u_0 - u_m) from the 5-point stencil of both
  const bool l = i > 0, r = i < n - 1, d = j > 0, t = j < n - 1;
  auto wdiff = [&](const double* __restrict__ um) {
    auto dq = [&](int q) { return U[q] - um[q]; };
    const double e = ((l ? dq(p - 1) : 0.0) + (r ? dq(p + 1) : 0.0)) + ((d ? dq(p - n) : 0.0) + (t ? dq(p + n) : 0.0));
    return fma(8.0, dq(p), e) * (1.0 / 12.0);
  };
#pragma unroll
  for (int m = 1; m < P; ++m) Rho[(size_t)(m - 1) * N + p] = wdiff(U + (size_t)m * N) + qf[m];
#pragma unroll
  for (int m = 0; m < P - 1; ++m) {
    const double sf = m == 0 ? qf[1] : qf[m + 1] - qf[m];
    // W f^E(u_m) = f~_m - nu L_9 u_m
    C[m * N + p] = fma(-tb.dtm[m], (ft[m] - g[m]) + g[m + 1], sf);
  }
}

// One damped-free Jacobi step for W r = rho on `count` arrays at once
// (blockIdx.z = array): r_out = (3/2) rho - (1/8) E(r_in), i.e.
// r <- D^{-1} (rho - (W - D) r) with D = 2/3; r_in == nullptr starts from 0.
// The iteration matrix -(1/8) E has max-norm 1/2, so every step halves the
// max-norm error.
__global__ void __launch_bounds__(kBX* kBY)
    k_winv_jacobi(int n, size_t N, const double* __restrict__ rho, const double* __restrict__ rin,
                  double* __restrict__ rout) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t base = size_t(blockIdx.z) * N;
  const int p = i + n * j;
  const double e = rin ? nbsum<double, 2>(rin + base, i, j, 0, n, p) : 0.0;
  rout[base + p] = fma(-0.125, e, 1.5 * rho[base + p]);
}

// One Chebyshev semi-iteration step for the same system (Golub-Varga, for
// y = T y + c with the spectrum of T = -(1/8) E inside [-1/2, 1/2]):
//   y_{k+1} = omega (T y_k + c - y_{k-1}) + y_{k-1},  c = (3/2) rho,
// with y_{k-1} = 0 when yprev == nullptr.  yout may be yprev (every point
// reads its own y_{k-1} before writing it).
__global__ void __launch_bounds__(kBX* kBY)
    k_winv_cheb(int n, size_t N, double omega, const double* __restrict__ rho, const double* __restrict__ ycur,
                const double* yprev, double* yout) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t base = size_t(blockIdx.z) * N;
  const int p = i + n * j;
  const double jac = fma(-0.125, nbsum<double, 2>(ycur + base, i, j, 0, n, p), 1.5 * rho[base + p]);
  const double yp = yprev ? yprev[base + p] : 0.0;
  yout[base + p] = fma(omega, jac - yp, yp);
}

// Max-norm over total values (grid-stride), integer max of the bit patterns.
__global__ void __launch_bounds__(256) k_maxabs(size_t total, const double* __restrict__ v,
                                                unsigned long long* __restrict__ out) {
  grid_dep_wait();
  unsigned long long rb = 0;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < total; q += size_t(gridDim.x) * blockDim.x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v[q]) & 0x7fffffffffffffffull;
    rb = bits > rb ? bits : rb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, rb, o);
    rb = w > rb ? w : rb;
  }
  if ((threadIdx.x & 31) == 0 && rb) atomicMax(out, rb);
}

// Gauss-Legendre end with the compact stencil, part 1: y = sum_j dt w_j nu L_9 u_j
// (the W^{-1} of it follows by k_winv_jacobi), part 2 below.
__global__ void __launch_bounds__(kBX* kBY)
    k_gauss_end9_sum(int n, size_t N, EndWeights ew, const double* __restrict__ G, double* __restrict__ y) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  double acc = ew.dtw[0] * G[N + p];
#pragma unroll
  for (int m = 1; m < kMaxM; ++m)
    if (m < ew.M) acc = fma(ew.dtw[m], G[(m + 1) * N + p], acc);
  y[p] = acc;
}

// Part 2: u = u_0 + sum_j dt w_j f^E(u_j) + W^{-1} y.
__global__ void __launch_bounds__(kBX* kBY)
    k_gauss_end9(int n, size_t N, EndWeights ew, int reaction, const double* __restrict__ U,
                 const double* __restrict__ winv_y, double* __restrict__ u) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= n) return;
  const int p = i + n * j;
  double acc = winv_y[p];
#pragma unroll
  for (int m = 0; m < kMaxM; ++m)
    if (m < ew.M) acc = fma(ew.dtw[m], reaction_term(reaction, U[(m + 1) * N + p]), acc);
  u[p] = U[p] + acc;
}

}  // namespace isdc
