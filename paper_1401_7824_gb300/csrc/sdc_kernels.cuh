// sdc_kernels.cuh -- sm_103a device kernels of the SDC sweep (FP64): spread,
// right-hand sides (Sec. 2, Eq. 4), the sweep end with the SDC residual
// (Sec. 3) and the Gauss-Legendre end quadrature.  The multigrid kernels are
// in kernels.cuh.
#pragma once
#include "kernels.cuh"

namespace isdc {

constexpr int kMaxM = 7;
constexpr int kMaxP = kMaxM + 1;

// Collocation tables premultiplied by dt (Sec. 2, Eq. 2), over the P points of
// a sweep: t_0 = T_n and the M nodes (P = M for Gauss-Lobatto, whose first
// node is t_0; P = M + 1 for Gauss-Radau and Gauss-Legendre).  Node j is
// point j + OFF with OFF = P - M.
struct SweepTables {
  int M, P;
  double dtQ[kMaxP][kMaxM];   // dt * int_{t_0}^{t_p} l_j; row 0 is zero
  double dtm[kMaxP];          // dt_m = t_{m+1} - t_m between consecutive points
};

// Start of a step: every point u_m = u, f_m = f^E(u) + nu L_h u, and the
// explicit part fe_m = f^E(u) (stored so that the sweep end need not
// re-evaluate it).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_spread(int n, size_t N, double nu_h2, int reaction, int M, const double* __restrict__ u,
             double* __restrict__ U, double* __restrict__ F, double* __restrict__ FE) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = u[p];
  const double fe = reaction_term(reaction, up);
  const double f = fe + nu_h2 * (nbsum<double, DIM>(u, i, j, k, n, p) - double(2 * DIM) * up);
  for (int m = 0; m < M; ++m) {
    U[m * N + p] = up;
    F[m * N + p] = f;
    FE[m * N + p] = fe;
  }
}

// f_m = f(u_m) and fe_m = f^E(u_m) for one point (resume from given node values).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_eval_f(int n, double nu_h2, int reaction, const double* __restrict__ u, double* __restrict__ f,
             double* __restrict__ fe_out) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = u[p];
  const double fe = reaction_term(reaction, up);
  fe_out[p] = fe;
  f[p] = fe + nu_h2 * (nbsum<double, DIM>(u, i, j, k, n, p) - double(2 * DIM) * up);
}

// Right-hand side of node m's implicit Euler system (Eq. 4, implicit unknown
// moved to the left), stored row-scaled as beta = b / d:
//   b = u_m^{k+1} + dt_m f^E(u_m^{k+1}) + C_m,
//   C_m = dt sum_j s_{m,j} f(u_j^k) - dt_m f^E(u_m^k) - dt_m f^I(u_{m+1}^k)
// (C_m comes from the end of the previous sweep).  For m >= 1 the same pass
// stores f_m = f(u_m^{k+1}) and fe_m = f^E(u_m^{k+1}), which the residual, the
// sweep end and the next sweep need.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs(int n, double nu_h2, int reaction, double dtm, double inv_d, const double* __restrict__ Um,
          const double* __restrict__ Cm, double* __restrict__ beta, double* __restrict__ Fm,
          double* __restrict__ FEm) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  const double up = Um[p];
  const double fe = reaction_term(reaction, up);
  beta[p] = (fma(dtm, fe, up) + Cm[p]) * inv_d;
  if (Fm) {
    Fm[p] = fe + nu_h2 * (nbsum<double, DIM>(Um, i, j, k, n, p) - double(2 * DIM) * up);
    FEm[p] = fe;
  }
}

// Mixed precision with a fixed V-cycle count: the defect of node m's system at
// its initial guess x = u_{m+1}^k (Sec. 4.3).  With the sweep constant in the
// defect form
//   C'_m = dt sum_j s_{m,j} f(u_j^k) - dt_m f^E(u_m^k) - u_{m+1}^k
// the implicit terms of b and of (I - a L_h) x cancel (a L_h u_{m+1}^k =
// dt_m f^I(u_{m+1}^k)), so
//   r = b - (I - a L_h) u_{m+1}^k = u_m^{k+1} + dt_m f^E(u_m^{k+1}) + C'_m
// needs no stencil of u_{m+1}^k.  r / d is computed in FP64 and stored in FP32;
// for m >= 1 the same pass stores f_m = f(u_m^{k+1}) and fe_m = f^E(u_m^{k+1}).
template <int DIM>
__device__ __forceinline__ float rhs_defect_point(int i, int j, int k, int n, int p, double nu_h2, int reaction,
                                                  double dtm, double inv_d, const double* __restrict__ Um,
                                                  const double* __restrict__ Cm, double* __restrict__ Fm,
                                                  double* __restrict__ FEm) {
  const double up = Um[p];
  const double fe = reaction_term(reaction, up);
  if (Fm) {
    Fm[p] = fe + nu_h2 * (nbsum<double, DIM>(Um, i, j, k, n, p) - double(2 * DIM) * up);
    FEm[p] = fe;
  }
  return float((fma(dtm, fe, up) + Cm[p]) * inv_d);
}

template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs_defect(int n, double nu_h2, int reaction, double dtm, double inv_d, const double* __restrict__ Um,
                 const double* __restrict__ Cm, double* __restrict__ Fm, double* __restrict__ FEm,
                 float* __restrict__ r32) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  r32[p] = rhs_defect_point<DIM>(i, j, k, n, p, nu_h2, reaction, dtm, inv_d, Um, Cm, Fm, FEm);
}

// The same into the colour-split FP32 arrays: one thread per slot pair (points
// 2h and 2h+1 of a row, one of each colour).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_rhs_defect_split(int n, double nu_h2, int reaction, double dtm, double inv_d, const double* __restrict__ Um,
                       const double* __restrict__ Cm, double* __restrict__ Fm, double* __restrict__ FEm,
                       float* __restrict__ r0, float* __restrict__ r1) {
  grid_dep_wait();
  const int h = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  const int H = (n + 1) >> 1;
  if (h >= H || j >= n) return;
  const int c0 = (j + (DIM == 3 ? k : 0) + DIM) & 1;  // colour of the even point 2h
  const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
  const int i = 2 * h;
  const int p = lin<DIM>(i, j, k, n);
  (c0 ? r1 : r0)[slot] = rhs_defect_point<DIM>(i, j, k, n, p, nu_h2, reaction, dtm, inv_d, Um, Cm, Fm, FEm);
  if (i + 1 < n)
    (c0 ? r0 : r1)[slot] =
        rhs_defect_point<DIM>(i + 1, j, k, n, p + 1, nu_h2, reaction, dtm, inv_d, Um, Cm, Fm, FEm);
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
// and the sweep constants of the next sweep: C_m (cmode 0, the form k_rhs
// adds) or C'_m (cmode 1, the defect form of k_rhs_defect).  Node arrays are
// node-major with stride N.  *Rbits must be zero on entry.
template <int DIM, int OFF, int P>
__global__ void __launch_bounds__(kBX* kBY)
    k_sweep_end(int n, size_t N, double nu_h2, int reaction, int cmode, SweepTables tb,
                const double* __restrict__ U, double* __restrict__ F, const double* __restrict__ FE,
                double* __restrict__ C, unsigned long long* __restrict__ Rbits) {
  grid_dep_wait();
  constexpr int M = P - OFF;  // nodes; node j is point j + OFF
  static_assert(M >= 2 && M <= kMaxM && P <= kMaxP, "point count out of range");
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = lin<DIM>(i, j, k, n);
    double u[P], f[P], fe[P], qf[P];
#pragma unroll
    for (int m = 0; m < P; ++m) u[m] = U[m * N + p];
    // f^E of the points before the last was stored with their f (spread, right-hand sides)
#pragma unroll
    for (int m = 0; m < P - 1; ++m) fe[m] = FE[m * N + p];
    fe[P - 1] = reaction_term(reaction, u[P - 1]);
    // f at the last point from its stencil; the other nodes' f were stored during the sweep
    const double* ul = U + (size_t)(P - 1) * N;
    const double ulast = u[P - 1];
    const double flast = fe[P - 1] + nu_h2 * (nbsum<double, DIM>(ul, i, j, k, n, p) - double(2 * DIM) * ulast);
    F[(size_t)(P - 1) * N + p] = flast;
#pragma unroll
    for (int m = OFF; m < P - 1; ++m) f[m] = F[m * N + p];
    f[P - 1] = flast;
    // dt sum_j q_{m,j} f_j for the points m >= 1 (row 0 is zero); the
    // point-to-point term dt sum_j s_{m,j} f_j of Eq. 2 is the difference of
    // consecutive rows.
    qf[0] = 0.0;
#pragma unroll
    for (int m = 1; m < P; ++m) {
      double acc = tb.dtQ[m][0] * f[OFF];
#pragma unroll
      for (int jj = 1; jj < M; ++jj) acc = fma(tb.dtQ[m][jj], f[jj + OFF], acc);
      qf[m] = acc;
    }
    // max of |r| on the integer pipe: with the sign bit cleared, doubles order
    // like their bit patterns (NaN above Inf), so no FP64 compares are needed
#pragma unroll
    for (int m = 1; m < P; ++m) {
      const unsigned long long rbits =
          (unsigned long long)__double_as_longlong((u[0] - u[m]) + qf[m]) & 0x7fffffffffffffffull;
      rb = rbits > rb ? rbits : rb;
    }
#pragma unroll
    for (int m = 0; m < P - 1; ++m) {
      const double sf = m == 0 ? qf[1] : qf[m + 1] - qf[m];
      // f^I(u_{m+1}) = f_{m+1} - f^E(u_{m+1})
      C[m * N + p] = cmode ? fma(-tb.dtm[m], fe[m], sf) - u[m + 1]
                           : fma(-tb.dtm[m], fe[m] + (f[m + 1] - fe[m + 1]), sf);
    }
  }
  block_max_atomic(rb, Rbits);
}

// End of a Gauss-Legendre step (tau_M < 1): the collocation rule's full-step
// quadrature u = u_0 + dt sum_j w_j f(u_j) (Sec. 2), with u_0 in point 0 and
// f of node j in point j + 1.
struct EndWeights {
  int M;
  double dtw[kMaxM];  // dt * w_j, w_j = int_0^1 l_j
};

template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_gauss_end(int n, size_t N, EndWeights ew, const double* __restrict__ U, const double* __restrict__ F,
                double* __restrict__ u) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  double acc = ew.dtw[0] * F[N + p];
#pragma unroll
  for (int m = 1; m < kMaxM; ++m)
    if (m < ew.M) acc = fma(ew.dtw[m], F[(m + 1) * N + p], acc);
  u[p] = U[p] + acc;
}

// Max-norm of b - H x (classical SDC stopping test), FP64.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_resnorm(int n, double kappa, double d, const double* __restrict__ x, const double* __restrict__ beta,
              unsigned long long* __restrict__ out) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  unsigned long long rb = 0;
  if (i < n && j < n) {
    const int p = lin<DIM>(i, j, k, n);
    const double r = d * (fma(kappa, nbsum<double, DIM>(x, i, j, k, n, p), beta[p]) - x[p]);
    rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
  }
  block_max_atomic(rb, out);
}

}  // namespace isdc
