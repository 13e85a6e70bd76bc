// periodic_kernels.cuh -- sm_103a kernels of the viscous Burgers equation of
// Sec. 4.1 on a periodic grid: u_t + sum_axes u u_x = nu Lap u on [-1,1)^DIM,
// n = 2^j points per side (h = 2/n), x fastest, indices wrap (n is a power
// of two, so a wrap is a mask).  The Laplacian is implicit (periodic 5/7-point
// stencil, multigrid n, n/2, ..., 4 with a dense solve on the side-4 level);
// the advection is explicit: conservative differences of u^2/2 with the
// 5th-order WENO scheme of Jiang and Shu and local Lax-Friedrichs splitting
// (alpha = max |u| over the six points of each face's stencil).  Levels with
// side <= 32 (2D) / 8 (3D) run in one block (k_bottom_per).
#pragma once
#include "sdc_kernels.cuh"

namespace isdc {

template <int DIM>
__device__ __forceinline__ int plin(int i, int j, int k, int n) {
  return DIM == 2 ? i + n * j : i + n * (j + n * k);
}

// Sum of the 2*DIM neighbours of (i,j,k) on the periodic grid.
template <typename T, int DIM>
__device__ __forceinline__ T pnbsum(const T* __restrict__ x, int i, int j, int k, int n) {
  const int w = n - 1;
  const T sx = x[plin<DIM>((i - 1) & w, j, k, n)] + x[plin<DIM>((i + 1) & w, j, k, n)];
  const T sy = x[plin<DIM>(i, (j - 1) & w, k, n)] + x[plin<DIM>(i, (j + 1) & w, k, n)];
  if (DIM == 2) return sx + sy;
  const T sz = x[plin<DIM>(i, j, (k - 1) & w, n)] + x[plin<DIM>(i, j, (k + 1) & w, n)];
  return (sx + sy) + sz;
}

// ---------------------------------------------------------------------------
// Multigrid on the row-scaled periodic system x - kappa * (neighbour sum) = beta.
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_jacobi_per(int n, T kappa, T omega, const T* __restrict__ x, const T* __restrict__ beta, T* __restrict__ xo,
                 int zero_guess) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = plin<DIM>(i, j, k, n);
  if (zero_guess) {
    xo[p] = omega * beta[p];
    return;
  }
  const T xp = x[p];
  xo[p] = fma(omega, fma(kappa, pnbsum<T, DIM>(x, i, j, k, n), beta[p]) - xp, xp);
}

// Red-black half sweep, red = i+j(+k) even (0-based; n even keeps the
// colouring consistent across the wrap).  Grid over (n/2) x n (x n).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs_per(int n, T kappa, int colour, T* __restrict__ x, const T* __restrict__ beta, int zero_guess) {
  grid_dep_wait();
  const int ih = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (2 * ih >= n || j >= n) return;
  const int i = 2 * ih + ((colour + j + (DIM == 3 ? k : 0)) & 1);
  const int p = plin<DIM>(i, j, k, n);
  x[p] = zero_guess ? beta[p] : fma(kappa, pnbsum<T, DIM>(x, i, j, k, n), beta[p]);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_residual_per(int n, T kappa, const T* __restrict__ x, const T* __restrict__ beta, T* __restrict__ r) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = plin<DIM>(i, j, k, n);
  r[p] = fma(kappa, pnbsum<T, DIM>(x, i, j, k, n), beta[p]) - x[p];
}

// Full weighting to the coarse periodic grid (nc = n/2 points): coarse I sits
// on fine 2I; weights [1 2 1] per axis, times wscale = d_f / (2^(2 DIM) d_c).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_restrict_per(int nc, T wscale, const T* __restrict__ r, T* __restrict__ bc) {
  grid_dep_wait();
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y, K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  const int n = 2 * nc, w = n - 1;
  auto row = [&](int j, int k) {
    const T a = r[plin<DIM>((2 * I - 1) & w, j, k, n)], b = r[plin<DIM>(2 * I, j, k, n)],
            c = r[plin<DIM>((2 * I + 1) & w, j, k, n)];
    return (a + c) + T(2) * b;
  };
  auto plane = [&](int k) {
    return (row((2 * J - 1) & w, k) + row((2 * J + 1) & w, k)) + T(2) * row(2 * J, k);
  };
  T acc;
  if (DIM == 2) acc = plane(0);
  else acc = (plane((2 * K - 1) & w) + plane((2 * K + 1) & w)) + T(2) * plane(2 * K);
  bc[plin<DIM>(I, J, K, nc)] = acc * wscale;
}

// x += P e_c: linear interpolation from the coarse periodic grid, one thread
// per fine point (even index: the coarse point; odd: the mean of two).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_prolong_per(int nc, const T* __restrict__ ec, T* __restrict__ x) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const int n = 2 * nc, w = nc - 1;
  if (i >= n || j >= n) return;
  auto axis = [&](int f, int& c0, int& c1, T& w1) {  // coarse neighbours and the weight of the second
    c0 = f >> 1;
    c1 = (c0 + 1) & w;
    w1 = (f & 1) ? T(0.5) : T(0);
  };
  int i0, i1, j0, j1, k0 = 0, k1 = 0;
  T wi, wj, wk = T(0);
  axis(i, i0, i1, wi);
  axis(j, j0, j1, wj);
  if (DIM == 3) axis(k, k0, k1, wk);
  auto ev = [&](int kk) {
    const T a = ec[plin<DIM>(i0, j0, kk, nc)], b = ec[plin<DIM>(i1, j0, kk, nc)];
    const T c = ec[plin<DIM>(i0, j1, kk, nc)], d = ec[plin<DIM>(i1, j1, kk, nc)];
    const T lo = a + wi * (b - a), hi = c + wi * (d - c);
    return lo + wj * (hi - lo);
  };
  T v = ev(k0);
  if (DIM == 3) v = v + wk * (ev(k1) - v);
  x[plin<DIM>(i, j, k, n)] += v;
}

template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_resnorm_per(int n, double kappa, double d, const double* __restrict__ x, const double* __restrict__ beta,
                  unsigned long long* __restrict__ out) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = plin<DIM>(i, j, k, n);
    const double r = d * (fma(kappa, pnbsum<double, DIM>(x, i, j, k, n), beta[p]) - x[p]);
    rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
  }
  block_max_atomic(rb, out);
}

// Bottom of the periodic V-cycle: every level with side <= the threshold in
// one block, in shared memory (local levels 0..nlev-1; the last is the side-4
// grid solved with the precomputed d (I - a L)^{-1}).  The grid-wide kernels'
// arithmetic: damped Jacobi or red-black Gauss-Seidel, full weighting and
// linear interpolation with wrap-around.
struct BottomParamsPer {
  int nlev;
  int side[kMaxLevels];
  double kappa[kMaxLevels];   // c/d per level
  double rscale[kMaxLevels];  // restriction factor d_l / (2^(2 DIM) d_{l+1})
  int smoother, nu1, nu2;
  double omega;
  const double* G;  // d (I - a L)^{-1} on the side-4 grid, row-major
};

template <int DIM>
__device__ void btp_smooth(const BottomParamsPer& P, int l, double* x, const double* b, double* t, bool zero) {
  const int n = P.side[l], Np = DIM == 2 ? n * n : n * n * n;
  const double kappa = P.kappa[l];
  if (P.smoother == 0) {
    for (int p = threadIdx.x; p < Np; p += blockDim.x) t[p] = x[p];
    __syncthreads();
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      x[p] = zero ? P.omega * b[p]
                  : fma(P.omega, fma(kappa, pnbsum<double, DIM>(t, i, j, k, n), b[p]) - t[p], t[p]);
    }
    __syncthreads();
  } else {
    for (int colour = 0; colour < 2; ++colour) {
      for (int p = threadIdx.x; p < Np; p += blockDim.x) {
        const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
        if (((i + j + k) & 1) != colour) continue;
        x[p] = (zero && colour == 0) ? b[p] : fma(kappa, pnbsum<double, DIM>(x, i, j, k, n), b[p]);
      }
      __syncthreads();
    }
  }
}

template <int DIM>
__global__ void __launch_bounds__(kBottomThreads)
    k_bottom_per(BottomParamsPer P, const double* __restrict__ b_top, double* __restrict__ x_top, int load_x) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* base = reinterpret_cast<double*>(smem_raw);
  double *X[kMaxLevels], *B[kMaxLevels], *Tt[kMaxLevels];
  int off = 0;
  for (int l = 0; l < P.nlev; ++l) {
    const int n = P.side[l], Np = DIM == 2 ? n * n : n * n * n;
    X[l] = base + off; off += Np;
    B[l] = base + off; off += Np;
    Tt[l] = base + off; off += Np;
  }
  {
    const int n = P.side[0], Np = DIM == 2 ? n * n : n * n * n;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      B[0][p] = b_top[p];
      X[0][p] = load_x ? x_top[p] : 0.0;
    }
  }
  __syncthreads();
  const int last = P.nlev - 1;
  for (int l = 0; l < last; ++l) {
    const int n = P.side[l], nc = P.side[l + 1];
    const int Np = DIM == 2 ? n * n : n * n * n, Nc = DIM == 2 ? nc * nc : nc * nc * nc;
    for (int s = 0; s < P.nu1; ++s) btp_smooth<DIM>(P, l, X[l], B[l], Tt[l], s == 0 && (l > 0 || !load_x));
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      Tt[l][p] = fma(P.kappa[l], pnbsum<double, DIM>(X[l], i, j, k, n), B[l][p]) - X[l][p];
    }
    __syncthreads();
    const int w = n - 1;
    for (int q = threadIdx.x; q < Nc; q += blockDim.x) {
      const int I = q % nc, J = (q / nc) % nc, K = DIM == 3 ? q / (nc * nc) : 0;
      auto row = [&](int j, int k) {
        const double a = Tt[l][plin<DIM>((2 * I - 1) & w, j, k, n)], b = Tt[l][plin<DIM>(2 * I, j, k, n)],
                     c = Tt[l][plin<DIM>((2 * I + 1) & w, j, k, n)];
        return (a + c) + 2.0 * b;
      };
      auto plane = [&](int k) { return (row((2 * J - 1) & w, k) + row((2 * J + 1) & w, k)) + 2.0 * row(2 * J, k); };
      const double acc = DIM == 2 ? plane(0)
                                  : (plane((2 * K - 1) & w) + plane((2 * K + 1) & w)) + 2.0 * plane(2 * K);
      B[l + 1][q] = acc * P.rscale[l];
      X[l + 1][q] = 0.0;
    }
    __syncthreads();
  }
  {
    const int n = P.side[last], Np = DIM == 2 ? n * n : n * n * n;
    for (int r = threadIdx.x; r < Np; r += blockDim.x) {
      double acc = 0.0;
      for (int q = 0; q < Np; ++q) acc = fma(P.G[r * Np + q], B[last][q], acc);
      X[last][r] = acc;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const int n = P.side[l], nc = P.side[l + 1], Np = DIM == 2 ? n * n : n * n * n, w = nc - 1;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      const int i0 = i >> 1, i1 = (i0 + 1) & w, j0 = j >> 1, j1 = (j0 + 1) & w;
      const double wi = (i & 1) ? 0.5 : 0.0, wj = (j & 1) ? 0.5 : 0.0;
      const double* ec = X[l + 1];
      auto ev = [&](int kk) {
        const double a = ec[plin<DIM>(i0, j0, kk, nc)], b = ec[plin<DIM>(i1, j0, kk, nc)];
        const double c = ec[plin<DIM>(i0, j1, kk, nc)], d = ec[plin<DIM>(i1, j1, kk, nc)];
        const double lo = a + wi * (b - a), hi = c + wi * (d - c);
        return lo + wj * (hi - lo);
      };
      double v;
      if (DIM == 2) {
        v = ev(0);
      } else {
        const int k0 = k >> 1, k1 = (k0 + 1) & w;
        const double wk = (k & 1) ? 0.5 : 0.0;
        v = ev(k0);
        v = v + wk * (ev(k1) - v);
      }
      X[l][p] += v;
    }
    __syncthreads();
    for (int s = 0; s < P.nu2; ++s) btp_smooth<DIM>(P, l, X[l], B[l], Tt[l], false);
  }
  {
    const int n = P.side[0], Np = DIM == 2 ? n * n : n * n * n;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) x_top[p] = X[0][p];
  }
}

// ---------------------------------------------------------------------------
// WENO5 advection, FP64.
// ---------------------------------------------------------------------------
// Face value from the five upwind-biased values v0..v4 (v2, v3 beside the
// face): three 3-point candidates q_k, smoothness indicators b_k, nonlinear
// weights a_k = d_k / (eps + b_k)^2 from the linear weights d = (1/10, 6/10,
// 3/10), eps = 1e-6, and the value sum a_k q_k / sum a_k.  Computed with one
// division: multiplying every a_k by the product of the three (eps + b_j)^2
// leaves d_k times the two other squares.  The candidates are kept as 6 q_k and
// the indicators as 4 b_k (13/3 s^2 + t^2 instead of 13/12 s^2 + 1/4 t^2, with
// 4 eps); the factor 4 cancels in the ratio and the 6 is divided out at the end.
__device__ __forceinline__ double weno5(double v0, double v1, double v2, double v3, double v4) {
  const double q0 = fma(2.0, v0, fma(-7.0, v1, 11.0 * v2));
  const double q1 = fma(5.0, v2, fma(2.0, v3, -v1));
  const double q2 = fma(2.0, v2, fma(5.0, v3, -v4));
  const double s0 = fma(-2.0, v1, v0 + v2), t0 = fma(-4.0, v1, fma(3.0, v2, v0));
  const double s1 = fma(-2.0, v2, v1 + v3), t1 = v1 - v3;
  const double s2 = fma(-2.0, v3, v2 + v4), t2 = fma(3.0, v2, fma(-4.0, v3, v4));
  constexpr double c = 13.0 / 3.0, e4 = 4e-6;
  const double e0 = fma(c * s0, s0, fma(t0, t0, e4));
  const double e1 = fma(c * s1, s1, fma(t1, t1, e4));
  const double e2 = fma(c * s2, s2, fma(t2, t2, e4));
  const double E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
  const double w0 = E1 * E2, w1 = 6.0 * (E0 * E2), w2 = 3.0 * (E0 * E1);
  return fma(w0, q0, fma(w1, q1, w2 * q2)) / (6.0 * ((w0 + w1) + w2));
}

// Numerical flux of u^2/2 at the face between w[2] and w[3] from the six
// values w[0..5] along the axis (local Lax-Friedrichs splitting with alpha =
// max |w|, taken on the integer pipe: with the sign bit cleared, doubles order
// like their bit patterns).  f(+/-) = (w^2/2 +/- alpha w)/2 = w (w/4 +/- alpha/2).
__device__ __forceinline__ double weno_flux(const double (&w)[6]) {
  unsigned long long ab = 0;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(w[t]) & 0x7fffffffffffffffull;
    ab = bits > ab ? bits : ab;
  }
  const double half_alpha = 0.5 * __longlong_as_double((long long)ab);
  double fp[6], fm[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    fp[t] = w[t] * fma(0.25, w[t], half_alpha);
    fm[t] = w[t] * fma(0.25, w[t], -half_alpha);
  }
  return weno5(fp[0], fp[1], fp[2], fp[3], fp[4]) + weno5(fm[5], fm[4], fm[3], fm[2], fm[1]);
}

// f^E(u) = -sum_axes (F_{i+1/2} - F_{i-1/2}) / h at point (i,j,k) of the
// calling thread, for a kBX x kBY block tile in the x-y plane: the tile and a
// halo of 3 are staged in shared memory and every x- and y-face flux of the
// tile is computed once (33 x 8 + 9 x 32 faces for 256 points instead of 4 per
// point); the z-faces (3D) come from the thread's own column.  Every thread
// of the block must call it (it synchronises); the faces and their order of
// use are those of the point-wise form, so the result is the same bit for bit.
struct WenoTile {
  double u[kBY + 6][kBX + 6];
  double fx[kBY][kBX + 1];  // face between tile points c-1 and c of row r
  double fy[kBY + 1][kBX];  // face between tile rows r-1 and r of column c
};

template <int DIM>
__device__ __forceinline__ double burgers_fe(const double* __restrict__ u, int k, int n, double inv_h, WenoTile& S) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kBX + tx, w = n - 1;
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY;
  for (int q = tid; q < (kBY + 6) * (kBX + 6); q += kBX * kBY) {
    const int r = q / (kBX + 6), c = q % (kBX + 6);
    S.u[r][c] = u[plin<DIM>((i0 - 3 + c) & w, (j0 - 3 + r) & w, k, n)];
  }
  __syncthreads();
  for (int q = tid; q < kBY * (kBX + 1); q += kBX * kBY) {
    const int r = q / (kBX + 1), c = q % (kBX + 1);
    const double wv[6] = {S.u[r + 3][c], S.u[r + 3][c + 1], S.u[r + 3][c + 2],
                          S.u[r + 3][c + 3], S.u[r + 3][c + 4], S.u[r + 3][c + 5]};
    S.fx[r][c] = weno_flux(wv);
  }
  for (int q = tid; q < (kBY + 1) * kBX; q += kBX * kBY) {
    const int r = q / kBX, c = q % kBX;
    const double wv[6] = {S.u[r][c + 3], S.u[r + 1][c + 3], S.u[r + 2][c + 3],
                          S.u[r + 3][c + 3], S.u[r + 4][c + 3], S.u[r + 5][c + 3]};
    S.fy[r][c] = weno_flux(wv);
  }
  __syncthreads();
  double acc = 0.0;
  acc -= (S.fx[ty][tx + 1] - S.fx[ty][tx]) * inv_h;
  acc -= (S.fy[ty + 1][tx] - S.fy[ty][tx]) * inv_h;
  if (DIM == 3) {
    const int i = (i0 + tx) & w, j = (j0 + ty) & w;
    double v[7];  // points k-3..k+3
#pragma unroll
    for (int t = 0; t < 7; ++t) v[t] = u[plin<DIM>(i, j, (k + t - 3) & w, n)];
    const double wr[6] = {v[1], v[2], v[3], v[4], v[5], v[6]};
    const double wl[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
    acc -= (weno_flux(wr) - weno_flux(wl)) * inv_h;
  }
  __syncthreads();  // S is reused by the next call
  return acc;
}

// ---------------------------------------------------------------------------
// SDC sweep for Burgers, FP64.  Per point p: U_p, F_p = f(u_p) and the
// explicit part FE_p = f^E(u_p) (stored: it is a wide stencil, not pointwise).
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double plap_part(const double* __restrict__ u, int i, int j, int k, int n, int p,
                                            double nu_h2) {
  return nu_h2 * (pnbsum<double, DIM>(u, i, j, k, n) - double(2 * DIM) * u[p]);
}

// Start of a step: every point u_p = u, FE_p = f^E(u), F_p = FE_p + nu L u.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_spread_b(int n, size_t N, double nu_h2, double inv_h, int P, const double* __restrict__ u,
               double* __restrict__ U, double* __restrict__ F, double* __restrict__ FE) {
  grid_dep_wait();
  __shared__ WenoTile S;
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const double fe = burgers_fe<DIM>(u, k, n, inv_h, S);  // every thread of the block takes part
  if (i >= n || j >= n) return;
  const int p = plin<DIM>(i, j, k, n);
  const double f = fe + plap_part<DIM>(u, i, j, k, n, p, nu_h2);
  const double up = u[p];
  for (int m = 0; m < P; ++m) {
    U[m * N + p] = up;
    F[m * N + p] = f;
    FE[m * N + p] = fe;
  }
}

// F and FE of one point's values (resume from given node values).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_eval_f_b(int n, double nu_h2, double inv_h, const double* __restrict__ u, double* __restrict__ f,
               double* __restrict__ fe) {
  grid_dep_wait();
  __shared__ WenoTile S;
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const double e = burgers_fe<DIM>(u, k, n, inv_h, S);
  if (i >= n || j >= n) return;
  const int p = plin<DIM>(i, j, k, n);
  fe[p] = e;
  f[p] = e + plap_part<DIM>(u, i, j, k, n, p, nu_h2);
}

// Right-hand side of node m's implicit Euler system (Eq. 4), row-scaled:
//   b = u_m^{k+1} + dt_m f^E(u_m^{k+1}) + C_m,
//   C_m = dt sum_j s_{m,j} f_j^k - dt_m f^E(u_m^k) - dt_m f^I(u_{m+1}^k).
// For m >= 1 f^E(u_m^{k+1}) is evaluated here and stored with f_m; for m = 0
// (u_0, fixed during the step) it is the stored value.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs_b(int n, double nu_h2, double inv_h, double dtm, double inv_d, const double* __restrict__ Um,
            const double* __restrict__ Cm, double* __restrict__ beta, double* __restrict__ Fm,
            double* __restrict__ FEm, int fresh) {
  grid_dep_wait();
  __shared__ WenoTile S;
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const double fnew = fresh ? burgers_fe<DIM>(Um, k, n, inv_h, S) : 0.0;  // fresh is uniform
  if (i >= n || j >= n) return;
  const int p = plin<DIM>(i, j, k, n);
  const double up = Um[p];
  double fe;
  if (fresh) {
    fe = fnew;
    FEm[p] = fe;
    Fm[p] = fe + plap_part<DIM>(Um, i, j, k, n, p, nu_h2);
  } else {
    fe = FEm[p];
  }
  beta[p] = (fma(dtm, fe, up) + Cm[p]) * inv_d;
}

// End of a sweep: f and f^E at the last point, the max-norm SDC residual
// (Sec. 3) and the next sweep's C_m.  Node j is point j + OFF.
template <int DIM, int OFF, int P>
__global__ void __launch_bounds__(kBX* kBY)
    k_sweep_end_b(int n, size_t N, double nu_h2, double inv_h, SweepTables tb, const double* __restrict__ U,
                  double* __restrict__ F, double* __restrict__ FE, double* __restrict__ C,
                  unsigned long long* __restrict__ Rbits) {
  grid_dep_wait();
  constexpr int M = P - OFF;
  static_assert(M >= 2 && M <= kMaxM && P <= kMaxP, "point count out of range");
  __shared__ WenoTile S;
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, k = blockIdx.z;
  const double* ul = U + (size_t)(P - 1) * N;
  const double fe_last = burgers_fe<DIM>(ul, k, n, inv_h, S);  // every thread of the block takes part
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = plin<DIM>(i, j, k, n);
    double u[P], f[P], fe[P], qf[P];
#pragma unroll
    for (int m = 0; m < P; ++m) u[m] = U[m * N + p];
    fe[P - 1] = fe_last;
    f[P - 1] = fe[P - 1] + plap_part<DIM>(ul, i, j, k, n, p, nu_h2);
    F[(size_t)(P - 1) * N + p] = f[P - 1];
    FE[(size_t)(P - 1) * N + p] = fe[P - 1];
#pragma unroll
    for (int m = 0; m < P - 1; ++m) {
      f[m] = F[m * N + p];
      fe[m] = FE[m * N + p];
    }
    qf[0] = 0.0;
#pragma unroll
    for (int m = 1; m < P; ++m) {
      double acc = tb.dtQ[m][0] * f[OFF];
#pragma unroll
      for (int jj = 1; jj < M; ++jj) acc = fma(tb.dtQ[m][jj], f[jj + OFF], acc);
      qf[m] = acc;
      const unsigned long long bits =
          (unsigned long long)__double_as_longlong((u[0] - u[m]) + acc) & 0x7fffffffffffffffull;
      rb = bits > rb ? bits : rb;
    }
#pragma unroll
    for (int m = 0; m < P - 1; ++m) {
      const double sf = m == 0 ? qf[1] : qf[m + 1] - qf[m];
      C[m * N + p] = fma(-tb.dtm[m], fe[m] + (f[m + 1] - fe[m + 1]), sf);
    }
  }
  block_max_atomic(rb, Rbits);
}

}  // namespace isdc
