// kernels.cuh -- sm_103a device kernels for the ISDC hot path.
//
// Grid arrays hold interior points only, x fastest: p = i + n*(j + n*k),
// 0-based i, j, k in [0, n); the zero Dirichlet ghosts are implicit.  The
// implicit operator of every node solve is H = I - a L_h (Sec. 3, Eq. 4 with
// W = I and A = nu L_h, a = dt_m nu); with c = a/h^2 and d = 1 + 2*DIM*c,
// H x = d x - c * (sum of the 2*DIM neighbours).
//
// Every kernel here is memory- or FP64-issue-bound stencil work on CUDA cores:
// no tensor cores (there is no dense contraction on this path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isdc {

constexpr int kBX = 32;  // threads along x (one warp)
constexpr int kBY = 8;   // rows per block

template <int DIM>
__device__ __forceinline__ int lin(int i, int j, int k, int n) {
  return DIM == 2 ? i + n * j : i + n * (j + n * k);
}

// Sum of the 2*DIM neighbours of (i,j,k); zero outside the interior.
template <typename T, int DIM>
__device__ __forceinline__ T nbsum(const T* __restrict__ x, int i, int j, int k, int n, int p) {
  const int sy = n, sz = n * n;
  T s = (i > 0 ? x[p - 1] : T(0)) + (i < n - 1 ? x[p + 1] : T(0));
  s += (j > 0 ? x[p - sy] : T(0));
  s += (j < n - 1 ? x[p + sy] : T(0));
  if (DIM == 3) {
    s += (k > 0 ? x[p - sz] : T(0));
    s += (k < n - 1 ? x[p + sz] : T(0));
  }
  return s;
}

template <typename T>
__device__ __forceinline__ T reaction_term(int reaction, T u) {
  // f^E(u) = u - u^3 (Allen-Cahn type) or nothing
  return reaction ? u - u * u * u : T(0);
}

// ---------------------------------------------------------------------------
// Multigrid smoothers, residual and transfers (one thread per point).
// ---------------------------------------------------------------------------

// Damped Jacobi: xo = x + (omega/d) (b - H x).  zero_guess: x == 0.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_jacobi(int n, T c, T d, T w_over_d, const T* __restrict__ x, const T* __restrict__ b,
             T* __restrict__ xo, int zero_guess) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  if (zero_guess) {
    xo[p] = w_over_d * b[p];
    return;
  }
  const T xp = x[p];
  const T r = b[p] - (d * xp - c * nbsum<T, DIM>(x, i, j, k, n, p));
  xo[p] = xp + w_over_d * r;
}

// Red-black Gauss-Seidel half sweep: colour 0 = red = (i+j+k) even in 1-based
// interior indices.  Each thread owns one point of the colour:
// x_p = (b_p + c * sum of neighbours) / d.  zero_guess (red pass from x == 0):
// the neighbours are zero.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs(int n, T c_over_d, T inv_d, int colour, T* __restrict__ x, const T* __restrict__ b,
           int zero_guess) {
  const int ih = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  // (i+1)+(j+1)+(k+1) parity == colour  <=>  i parity == (colour + j + k + DIM) & 1
  const int i = 2 * ih + ((colour + j + (DIM == 3 ? k : 0) + DIM) & 1);
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  if (zero_guess) {
    x[p] = inv_d * b[p];
    return;
  }
  x[p] = inv_d * b[p] + c_over_d * nbsum<T, DIM>(x, i, j, k, n, p);
}

// r = b - H x
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_residual(int n, T c, T d, const T* __restrict__ x, const T* __restrict__ b,
               T* __restrict__ r) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  r[p] = b[p] - (d * x[p] - c * nbsum<T, DIM>(x, i, j, k, n, p));
}

// Full weighting to the coarse grid (side nc, fine side 2nc+1): coarse point
// I sits on fine point 2I+1 (0-based); weights (1/4, 1/2, 1/4) per axis.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_restrict(int nc, const T* __restrict__ r, T* __restrict__ bc) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  const int n = 2 * nc + 1;
  const int fi = 2 * I + 1, fj = 2 * J + 1;
  T acc = T(0);
  if (DIM == 2) {
    T row[3];
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const T* q = r + (fi + n * (fj + dj));
      row[dj + 1] = (q[-1] + q[1]) + T(2) * q[0];
    }
    acc = ((row[0] + row[2]) + T(2) * row[1]) * T(1.0 / 16.0);
  } else {
    const int fk = 2 * K + 1;
    T pl[3];
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      T row[3];
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const T* q = r + (fi + n * ((fj + dj) + n * (fk + dk)));
        row[dj + 1] = (q[-1] + q[1]) + T(2) * q[0];
      }
      pl[dk + 1] = (row[0] + row[2]) + T(2) * row[1];
    }
    acc = ((pl[0] + pl[2]) + T(2) * pl[1]) * T(1.0 / 64.0);
  }
  bc[lin<DIM>(I, J, K, nc)] = acc;
}

// x += P e_c: (bi/tri)linear interpolation from the coarse grid (side nc) to
// the fine grid (side 2nc+1); coarse ghosts are zero.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_prolong_add(int nc, const T* __restrict__ ec, T* __restrict__ x) {
  const int n = 2 * nc + 1;
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  // fine 0-based i sits on coarse (i-1)/2 when i is odd; between (i-2)/2 and i/2 when even
  int ci[2], cj[2], ck[2];
  T wi[2], wj[2], wk[2];
  int ni, nj, nk;
  auto axis = [nc](int f, int* c, T* w, int* cnt) {
    if (f & 1) {
      c[0] = (f - 1) >> 1; w[0] = T(1); *cnt = 1;
    } else {
      int m = 0;
      if (f > 0) { c[m] = (f - 2) >> 1; w[m] = T(0.5); ++m; }
      if (f / 2 < nc) { c[m] = f >> 1; w[m] = T(0.5); ++m; }
      *cnt = m;
    }
  };
  axis(i, ci, wi, &ni);
  axis(j, cj, wj, &nj);
  if (DIM == 3) axis(k, ck, wk, &nk); else { ck[0] = 0; wk[0] = T(1); nk = 1; }
  T e = T(0);
  for (int c3 = 0; c3 < nk; ++c3)
    for (int c2 = 0; c2 < nj; ++c2) {
      T line = T(0);
      for (int c1 = 0; c1 < ni; ++c1) line += wi[c1] * ec[lin<DIM>(ci[c1], cj[c2], ck[c3], nc)];
      e += (wj[c2] * wk[c3]) * line;
    }
  x[lin<DIM>(i, j, k, n)] += e;
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 defect to FP32, FP32 correction added in FP64.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_defect(int n, double c, double d, const double* __restrict__ x,
             const double* __restrict__ b, float* __restrict__ r32) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  r32[p] = float(b[p] - (d * x[p] - c * nbsum<double, DIM>(x, i, j, k, n, p)));
}

template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_update(int n, double* __restrict__ x, const float* __restrict__ e32) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  x[p] += double(e32[p]);
}

// ---------------------------------------------------------------------------
// SDC kernels (FP64).
// ---------------------------------------------------------------------------
constexpr int kMaxM = 7;

// Collocation tables premultiplied by dt (Sec. 2, Eq. 2).
struct SweepTables {
  int M;
  double dtQ[kMaxM][kMaxM];   // dt * Q[m][j]
  double dtS[kMaxM][kMaxM];   // dt * S[m][j], rows m = 0..M-2
  double dtm[kMaxM];          // dt_m = dt (tau_{m+1} - tau_m)
};

// Start of a step: every node u_m = u, f_m = f^E(u) + nu L_h u.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_spread(int n, size_t N, double nu_h2, int reaction, int M, const double* __restrict__ u,
             double* __restrict__ U, double* __restrict__ F) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = u[p];
  const double f = reaction_term(reaction, up) +
                   nu_h2 * (nbsum<double, DIM>(u, i, j, k, n, p) - double(2 * DIM) * up);
  for (int m = 0; m < M; ++m) {
    U[m * N + p] = up;
    F[m * N + p] = f;
  }
}

// f_m = f(u_m) for one node (resume from given node values).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_eval_f(int n, double nu_h2, int reaction, const double* __restrict__ u, double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = u[p];
  f[p] = reaction_term(reaction, up) +
         nu_h2 * (nbsum<double, DIM>(u, i, j, k, n, p) - double(2 * DIM) * up);
}

// Right-hand side of node m's implicit Euler system (Eq. 4, implicit unknown
// moved to the left):
//   b = u_m^{k+1} + dt_m f^E(u_m^{k+1}) + C_m,
//   C_m = dt sum_j s_{m,j} f(u_j^k) - dt_m f^E(u_m^k) - dt_m f^I(u_{m+1}^k)
// (C_m comes from the end of the previous sweep).  For m >= 1 the same pass
// stores f_m = f(u_m^{k+1}), which the residual and the next sweep need.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs(int n, double nu_h2, int reaction, double dtm, const double* __restrict__ Um,
          const double* __restrict__ Cm, double* __restrict__ b, double* __restrict__ Fm) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = Um[p];
  const double fe = reaction_term(reaction, up);
  b[p] = up + dtm * fe + Cm[p];
  if (Fm) Fm[p] = fe + nu_h2 * (nbsum<double, DIM>(Um, i, j, k, n, p) - double(2 * DIM) * up);
}

__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long* out) {
  // Non-negative doubles order like their bit patterns; NaN sorts above Inf.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __shared__ unsigned long long wmax[kBX * kBY / 32];
  const int lane = (threadIdx.y * kBX + threadIdx.x) & 31, warp = (threadIdx.y * kBX + threadIdx.x) >> 5;
  if (lane == 0) wmax[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kBX * kBY / 32 ? wmax[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (lane == 0 && v) atomicMax(out, v);
  }
}

// End of a sweep: f_{M-1} = f(u_{M-1}), the SDC residual
//   R = max_m max_x | u_0 + dt sum_j q_{m,j} f_j - u_m |         (Sec. 3)
// and the sweep constants C_m of the next sweep.  Node arrays are node-major
// with stride N.  *Rbits must be zero on entry.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_sweep_end(int n, size_t N, double nu_h2, int reaction, SweepTables tb,
                const double* __restrict__ U, double* __restrict__ F, double* __restrict__ C,
                unsigned long long* __restrict__ Rbits) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = lin<DIM>(i, j, k, n);
    const int M = tb.M;
    double u[kMaxM], f[kMaxM], fe[kMaxM], qf[kMaxM];
#pragma unroll
    for (int m = 0; m < kMaxM; ++m)
      if (m < M) {
        u[m] = U[m * N + p];
        fe[m] = reaction_term(reaction, u[m]);
      }
    // f at the last node from its stencil; the other f_m were stored during the sweep
    const double* ul = U + (size_t)(M - 1) * N;
    const double ulast = ul[p];
    const double flast = reaction_term(reaction, ulast) +
                         nu_h2 * (nbsum<double, DIM>(ul, i, j, k, n, p) - double(2 * DIM) * ulast);
    F[(size_t)(M - 1) * N + p] = flast;
#pragma unroll
    for (int m = 0; m < kMaxM; ++m) {
      if (m < M - 1) f[m] = F[m * N + p];
      else if (m == M - 1) f[m] = flast;
    }
    double rmax = 0.0;
#pragma unroll
    for (int m = 0; m < kMaxM; ++m)
      if (m < M) {
        double acc = 0.0;
#pragma unroll
        for (int jj = 0; jj < kMaxM; ++jj)
          if (jj < M) acc += tb.dtQ[m][jj] * f[jj];
        qf[m] = acc;
        const double r = fabs(u[0] + acc - u[m]);
        rmax = (r > rmax || r != r) ? r : rmax;
      }
#pragma unroll
    for (int m = 0; m < kMaxM - 1; ++m)
      if (m < M - 1) {
        double sf = 0.0;
#pragma unroll
        for (int jj = 0; jj < kMaxM; ++jj)
          if (jj < M) sf += tb.dtS[m][jj] * f[jj];
        // f^I(u_{m+1}) = f_{m+1} - f^E(u_{m+1})
        C[m * N + p] = sf - tb.dtm[m] * (fe[m] + (f[m + 1] - fe[m + 1]));
      }
    rb = (unsigned long long)__double_as_longlong(rmax);
  }
  block_max_atomic(rb, Rbits);
}

// Max-norm of b - H x (classical SDC stopping test), FP64.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_resnorm(int n, double c, double d, const double* __restrict__ x, const double* __restrict__ b,
              unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = lin<DIM>(i, j, k, n);
    const double r = fabs(b[p] - (d * x[p] - c * nbsum<double, DIM>(x, i, j, k, n, p)));
    rb = (unsigned long long)__double_as_longlong(r);
  }
  block_max_atomic(rb, out);
}

// ---------------------------------------------------------------------------
// Bottom of the V-cycle: every level with side <= the threshold, in one block,
// in shared memory.  Levels 0..nlev-1 here (local numbering), the last one is
// the side-3 grid solved exactly with a precomputed dense inverse.
// ---------------------------------------------------------------------------
constexpr int kBottomThreads = 512;
constexpr int kMaxLevels = 12;

template <typename T>
struct BottomParams {
  int nlev;
  int side[kMaxLevels];
  T c[kMaxLevels], d[kMaxLevels];
  int smoother, nu1, nu2;
  T omega;
  const T* Ainv;  // dense inverse of H on the side-3 grid, row-major
};

template <typename T, int DIM>
__device__ void bt_smooth(const BottomParams<T>& P, int l, T* x, const T* b, T* t) {
  const int n = P.side[l];
  const int Np = DIM == 2 ? n * n : n * n * n;
  const T c = P.c[l], d = P.d[l];
  if (P.smoother == 0) {
    for (int p = threadIdx.x; p < Np; p += blockDim.x) t[p] = x[p];
    __syncthreads();
    const T wd = P.omega / d;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      const T r = b[p] - (d * t[p] - c * nbsum<T, DIM>(t, i, j, k, n, p));
      x[p] = t[p] + wd * r;
    }
    __syncthreads();
  } else {
    const T cd = c / d, id = T(1) / d;
    for (int colour = 0; colour < 2; ++colour) {
      for (int p = threadIdx.x; p < Np; p += blockDim.x) {
        const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
        if (((i + j + k + DIM) & 1) != colour) continue;
        x[p] = id * b[p] + cd * nbsum<T, DIM>(x, i, j, k, n, p);
      }
      __syncthreads();
    }
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBottomThreads)
    k_bottom(BottomParams<T> P, const T* __restrict__ b_top, T* __restrict__ x_top, int load_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* base = reinterpret_cast<T*>(smem_raw);
  T *X[kMaxLevels], *B[kMaxLevels], *Tt[kMaxLevels];
  int off = 0;
  for (int l = 0; l < P.nlev; ++l) {
    const int n = P.side[l];
    const int Np = DIM == 2 ? n * n : n * n * n;
    X[l] = base + off; off += Np;
    B[l] = base + off; off += Np;
    Tt[l] = base + off; off += Np;
  }
  {
    const int n = P.side[0];
    const int Np = DIM == 2 ? n * n : n * n * n;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      B[0][p] = b_top[p];
      X[0][p] = load_x ? x_top[p] : T(0);
    }
  }
  __syncthreads();
  const int last = P.nlev - 1;
  // downward leg
  for (int l = 0; l < last; ++l) {
    const int n = P.side[l], nc = P.side[l + 1];
    const int Np = DIM == 2 ? n * n : n * n * n;
    const int Nc = DIM == 2 ? nc * nc : nc * nc * nc;
    for (int s = 0; s < P.nu1; ++s) bt_smooth<T, DIM>(P, l, X[l], B[l], Tt[l]);
    const T c = P.c[l], d = P.d[l];
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      Tt[l][p] = B[l][p] - (d * X[l][p] - c * nbsum<T, DIM>(X[l], i, j, k, n, p));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Nc; q += blockDim.x) {
      const int I = q % nc, J = (q / nc) % nc, K = DIM == 3 ? q / (nc * nc) : 0;
      const int fi = 2 * I + 1, fj = 2 * J + 1, fk = 2 * K + 1;
      T acc;
      if (DIM == 2) {
        T row[3];
        for (int dj = -1; dj <= 1; ++dj) {
          const T* r = Tt[l] + (fi + n * (fj + dj));
          row[dj + 1] = (r[-1] + r[1]) + T(2) * r[0];
        }
        acc = ((row[0] + row[2]) + T(2) * row[1]) * T(1.0 / 16.0);
      } else {
        T pl[3];
        for (int dk = -1; dk <= 1; ++dk) {
          T row[3];
          for (int dj = -1; dj <= 1; ++dj) {
            const T* r = Tt[l] + (fi + n * ((fj + dj) + n * (fk + dk)));
            row[dj + 1] = (r[-1] + r[1]) + T(2) * r[0];
          }
          pl[dk + 1] = (row[0] + row[2]) + T(2) * row[1];
        }
        acc = ((pl[0] + pl[2]) + T(2) * pl[1]) * T(1.0 / 64.0);
      }
      B[l + 1][q] = acc;
      X[l + 1][q] = T(0);
    }
    __syncthreads();
  }
  // coarsest grid: x = H^{-1} b with the precomputed dense inverse
  {
    const int n = P.side[last];
    const int Np = DIM == 2 ? n * n : n * n * n;
    for (int r = threadIdx.x; r < Np; r += blockDim.x) {
      T acc = T(0);
      for (int q = 0; q < Np; ++q) acc += P.Ainv[r * Np + q] * B[last][q];
      X[last][r] = acc;
    }
    __syncthreads();
  }
  // upward leg
  for (int l = last - 1; l >= 0; --l) {
    const int n = P.side[l], nc = P.side[l + 1];
    const int Np = DIM == 2 ? n * n : n * n * n;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      int ci[2], cj[2], ck[2];
      T wi[2], wj[2], wk[2];
      int ni = 0, nj = 0, nk = 0;
      auto axis = [nc](int f, int* cc, T* w, int* cnt) {
        if (f & 1) {
          cc[0] = (f - 1) >> 1; w[0] = T(1); *cnt = 1;
        } else {
          int m = 0;
          if (f > 0) { cc[m] = (f - 2) >> 1; w[m] = T(0.5); ++m; }
          if (f / 2 < nc) { cc[m] = f >> 1; w[m] = T(0.5); ++m; }
          *cnt = m;
        }
      };
      axis(i, ci, wi, &ni);
      axis(j, cj, wj, &nj);
      if (DIM == 3) axis(k, ck, wk, &nk); else { ck[0] = 0; wk[0] = T(1); nk = 1; }
      T e = T(0);
      for (int c3 = 0; c3 < nk; ++c3)
        for (int c2 = 0; c2 < nj; ++c2) {
          T line = T(0);
          for (int c1 = 0; c1 < ni; ++c1) line += wi[c1] * X[l + 1][lin<DIM>(ci[c1], cj[c2], ck[c3], nc)];
          e += (wj[c2] * wk[c3]) * line;
        }
      X[l][p] += e;
    }
    __syncthreads();
    for (int s = 0; s < P.nu2; ++s) bt_smooth<T, DIM>(P, l, X[l], B[l], Tt[l]);
  }
  {
    const int n = P.side[0];
    const int Np = DIM == 2 ? n * n : n * n * n;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) x_top[p] = X[0][p];
  }
}

}  // namespace isdc
