// kernels.cuh -- sm_103a device kernels for the ISDC hot path.
//
// Grid arrays hold interior points only, x fastest: p = i + n*(j + n*k),
// 0-based i, j, k in [0, n); the zero Dirichlet ghosts are implicit.  The
// implicit operator of every node solve is H = I - a L_h (Sec. 3, Eq. 4 with
// W = I and A = nu L_h, a = dt_m nu); with c = a/h^2 and d = 1 + 2*DIM*c,
// H x = d x - c * (sum of the 2*DIM neighbours).  The multigrid kernels work on
// the row-scaled system x - kappa * (neighbour sum) = beta, kappa = c/d,
// beta = b/d, so a Gauss-Seidel update is one FMA after the neighbour sum.
//
// Every kernel here is memory- or FP64-issue-bound stencil work on CUDA cores:
// no tensor cores (there is no dense contraction on this path).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isdc {

// Entry of every kernel: when the kernel was launched through a programmatic
// edge of a replayed graph (its launch overlapping the end of the kernel before
// it), wait until that kernel has completed and its writes are visible; after
// an ordinary launch this returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr int kBX = 32;  // threads along x (one warp)
constexpr int kBY = 8;   // rows per block

template <int DIM>
__device__ __forceinline__ int lin(int i, int j, int k, int n) {
  return DIM == 2 ? i + n * j : i + n * (j + n * k);
}

// Sum of the 2*DIM neighbours of (i,j,k); zero outside the interior.  Summed
// as a tree (pairs per axis) for short FP64 dependency chains.
template <typename T, int DIM>
__device__ __forceinline__ T nbsum(const T* __restrict__ x, int i, int j, int k, int n, int p) {
  const int sy = n, sz = n * n;
  const T sx = (i > 0 ? x[p - 1] : T(0)) + (i < n - 1 ? x[p + 1] : T(0));
  const T syv = (j > 0 ? x[p - sy] : T(0)) + (j < n - 1 ? x[p + sy] : T(0));
  if (DIM == 3) {
    const T szv = (k > 0 ? x[p - sz] : T(0)) + (k < n - 1 ? x[p + sz] : T(0));
    return (sx + syv) + szv;
  }
  return sx + syv;
}

template <typename T>
__device__ __forceinline__ T reaction_term(int reaction, T u) {
  // f^E(u) = u - u^3 (Allen-Cahn type) or nothing; one multiply + one FMA
  return reaction ? fma(-(u * u), u, u) : T(0);
}

// ---------------------------------------------------------------------------
// Multigrid smoothers, residual and transfers (one thread per point).
// ---------------------------------------------------------------------------

// Damped Jacobi: xo = x + omega (beta - x + kappa * sum) = x + (omega/d)(b - H x).
// zero_guess: x == 0.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_jacobi(int n, T kappa, T omega, const T* __restrict__ x, const T* __restrict__ beta,
             T* __restrict__ xo, int zero_guess) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  if (zero_guess) {
    xo[p] = omega * beta[p];
    return;
  }
  const T xp = x[p];
  xo[p] = fma(omega, fma(kappa, nbsum<T, DIM>(x, i, j, k, n, p), beta[p]) - xp, xp);
}

// Red-black Gauss-Seidel half sweep: colour 0 = red = (i+j+k) even in 1-based
// interior indices.  Each thread owns points of the colour and solves their
// rows: x_p = beta_p + kappa * (sum of neighbours).  zero_guess (red pass from
// x == 0): the neighbours are zero.  A colour pass reads only the other
// colour, so every thread issues all its loads before its first store.
//
// 2D: one point per thread.
template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs2(int n, T kappa, int colour, T* __restrict__ x, const T* __restrict__ beta, int zero_guess) {
  grid_dep_wait();
  const int ih = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (j >= n) return;
  // (i+1)+(j+1) parity == colour  <=>  i parity == (colour + j) & 1
  const int i = 2 * ih + ((colour + j) & 1);
  if (i >= n) return;
  const int p = lin<2>(i, j, 0, n);
  x[p] = zero_guess ? beta[p] : fma(kappa, nbsum<T, 2>(x, i, j, 0, n, p), beta[p]);
}

// 3D: each thread walks zb points of the colour along the (0,1,1) diagonal at
// a fixed i, p_t = (i, jd + t, k0 + t), t < zb (the colour of a point does not
// change along that diagonal).  The neighbour sum is built from three pair
// sums, X = x(i-1) + x(i+1), L = x(j-1) + x(k-1), U = x(j+1) + x(k+1), as
// (X + L) + U.  U at p_t is the sum of the same two points as L at p_{t+1},
// so a step loads 4 neighbours and issues 4 additions and one FMA where the
// plain sum takes 6 and 6.  The next step's loads are issued before the
// current store (they read the other colour).  Addition is commutative in
// IEEE arithmetic, so a point's value does not depend on zb or on where its
// diagonal starts.
template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs3(int n, T kappa, int colour, T* __restrict__ x, const T* __restrict__ beta, int zero_guess, int zb) {
  grid_dep_wait();
  const int ih = blockIdx.x * kBX + threadIdx.x;
  const int jd = int(blockIdx.y * kBY + threadIdx.y) - (zb - 1);
  const int k0 = blockIdx.z * zb;
  // (i+1)+(j+1)+(k+1) parity == colour, j + k = jd + k0 + 2t
  const int i = 2 * ih + ((colour + jd + k0 + 1) & 1);
  if (i >= n) return;
  const int t0 = jd < 0 ? -jd : 0, t1 = min(zb, min(n - jd, n - k0));
  if (t0 >= t1) return;
  const int nn = n * n, step = n + nn;
  int j = jd + t0, k = k0 + t0, p = i + n * j + nn * k;
  if (zero_guess) {
    for (int t = t0; t < t1; ++t, p += step) x[p] = beta[p];
    return;
  }
  const bool xl = i > 0, xr = i < n - 1;
  T lo = (j > 0 ? x[p - n] : T(0)) + (k > 0 ? x[p - nn] : T(0));
  T xs = (xl ? x[p - 1] : T(0)) + (xr ? x[p + 1] : T(0));
  T up = (j < n - 1 ? x[p + n] : T(0)) + (k < n - 1 ? x[p + nn] : T(0));
  T bp = beta[p];
  for (int t = t0; t < t1; ++t) {
    T xs1 = T(0), up1 = T(0), bp1 = T(0);
    if (t + 1 < t1) {
      const int q = p + step;
      xs1 = (xl ? x[q - 1] : T(0)) + (xr ? x[q + 1] : T(0));
      up1 = (j + 1 < n - 1 ? x[q + n] : T(0)) + (k + 1 < n - 1 ? x[q + nn] : T(0));
      bp1 = beta[q];
    }
    x[p] = fma(kappa, (xs + lo) + up, bp);
    lo = up;
    xs = xs1;
    up = up1;
    bp = bp1;
    p += step;
    ++j;
    ++k;
  }
}

// The same pass with the run length ZB fixed at compile time and all loads of
// the run issued before its first store (more loads in flight per thread, at
// more registers): the faster form where the pass is latency bound (small or
// FP32 levels).
template <typename T, int ZB>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs3_burst(int n, T kappa, int colour, T* __restrict__ x, const T* __restrict__ beta, int zero_guess) {
  grid_dep_wait();
  const int ih = blockIdx.x * kBX + threadIdx.x;
  const int jd = int(blockIdx.y * kBY + threadIdx.y) - (ZB - 1);
  const int k0 = blockIdx.z * ZB;
  // (i+1)+(j+1)+(k+1) parity == colour, j + k = jd + k0 + 2t
  const int i = 2 * ih + ((colour + jd + k0 + 1) & 1);
  if (i >= n) return;
  const int nn = n * n;
  T xs[ZB], us[ZB], bs[ZB], l0 = T(0);
#pragma unroll
  for (int t = 0; t < ZB; ++t) {
    const int j = jd + t, k = k0 + t;
    if (j < 0 || j >= n || k >= n) continue;
    const int p = i + n * j + nn * k;
    bs[t] = beta[p];
    if (zero_guess) continue;
    xs[t] = (i > 0 ? x[p - 1] : T(0)) + (i < n - 1 ? x[p + 1] : T(0));
    us[t] = (j < n - 1 ? x[p + n] : T(0)) + (k < n - 1 ? x[p + nn] : T(0));
    if (t == 0 || j == 0) l0 = (j > 0 ? x[p - n] : T(0)) + (k > 0 ? x[p - nn] : T(0));  // first point
  }
#pragma unroll
  for (int t = 0; t < ZB; ++t) {
    const int j = jd + t, k = k0 + t;
    if (j < 0 || j >= n || k >= n) continue;
    const int p = i + n * j + nn * k;
    if (zero_guess) {
      x[p] = bs[t];
      continue;
    }
    const T lt = (t == 0 || j == 0) ? l0 : us[t > 0 ? t - 1 : 0];
    x[p] = fma(kappa, (xs[t] + lt) + us[t], bs[t]);
  }
}

// One colour pass of the natural-layout red-black smoother.  zb: the 3D run
// length (the context's autotuner picks it); zb > 0 streams runs of zb points
// (k_rbgs3), zb in {-1, -2, -4, -8} issues runs of -zb points in one burst
// (k_rbgs3_burst).
template <typename T, int DIM>
inline void launch_rbgs(cudaStream_t st, int n, T kappa, int colour, T* x, const T* beta, bool zero_guess, int zb) {
  const dim3 blk(kBX, kBY, 1);
  const int gx = ((n + 1) / 2 + kBX - 1) / kBX;
  const int zg = zero_guess ? 1 : 0;
  if (DIM == 2) {
    k_rbgs2<T><<<dim3(gx, (n + kBY - 1) / kBY, 1), blk, 0, st>>>(n, kappa, colour, x, beta, zg);
    return;
  }
  const int run = zb < 0 ? -zb : zb;
  const dim3 g(gx, (n + run - 1 + kBY - 1) / kBY, (n + run - 1) / run);
  switch (zb) {
    case -1: k_rbgs3_burst<T, 1><<<g, blk, 0, st>>>(n, kappa, colour, x, beta, zg); break;
    case -2: k_rbgs3_burst<T, 2><<<g, blk, 0, st>>>(n, kappa, colour, x, beta, zg); break;
    case -4: k_rbgs3_burst<T, 4><<<g, blk, 0, st>>>(n, kappa, colour, x, beta, zg); break;
    case -8: k_rbgs3_burst<T, 8><<<g, blk, 0, st>>>(n, kappa, colour, x, beta, zg); break;
    default: k_rbgs3<T><<<g, blk, 0, st>>>(n, kappa, colour, x, beta, zg, run); break;
  }
}

// Scaled residual r' = beta - x + kappa * sum = (b - H x)/d.
// RED_ONLY (launched with the red-black grid): right after a complete
// red-black sweep every black row is satisfied, so only the red points carry
// a residual; the black entries of r are left unwritten and never read.
template <typename T, int DIM, bool RED_ONLY = false>
__global__ void __launch_bounds__(kBX* kBY)
    k_residual(int n, T kappa, const T* __restrict__ x, const T* __restrict__ beta, T* __restrict__ r) {
  grid_dep_wait();
  const int t = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  const int i = RED_ONLY ? 2 * t + ((j + (DIM == 3 ? k : 0) + DIM) & 1) : t;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  r[p] = fma(kappa, nbsum<T, DIM>(x, i, j, k, n, p), beta[p]) - x[p];
}

// Full weighting at coarse point (I,J,K) (see k_restrict).
// RED_ONLY: the residual vanishes at the black points (see k_residual); the
// coarse point's own fine point and its edge neighbours are red, its face and
// corner neighbours black, so full weighting keeps 5 (2D) or 13 (3D) terms.
template <typename T, int DIM, bool RED_ONLY>
__device__ __forceinline__ T restrict_point(int nc, T wscale, const T* __restrict__ r, int I, int J, int K) {
  const int n = 2 * nc + 1;
  const int fi = 2 * I + 1, fj = 2 * J + 1;
  if (RED_ONLY) {
    if (DIM == 2) {
      const T* q = r + (fi + n * fj);
      return fma(T(4), q[0], (q[-n - 1] + q[-n + 1]) + (q[n - 1] + q[n + 1])) * wscale;
    }
    const int nn = n * n;
    const T* q = r + (fi + n * (fj + n * (2 * K + 1)));
    const T e_xy = (q[-n - 1] + q[-n + 1]) + (q[n - 1] + q[n + 1]);
    const T e_xz = (q[-nn - 1] + q[-nn + 1]) + (q[nn - 1] + q[nn + 1]);
    const T e_yz = (q[-nn - n] + q[-nn + n]) + (q[nn - n] + q[nn + n]);
    return fma(T(2), (e_xy + e_xz) + e_yz, T(8) * q[0]) * wscale;
  }
  if (DIM == 2) {
    T row[3];
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const T* q = r + (fi + n * (fj + dj));
      row[dj + 1] = (q[-1] + q[1]) + T(2) * q[0];
    }
    return ((row[0] + row[2]) + T(2) * row[1]) * wscale;
  }
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
  return ((pl[0] + pl[2]) + T(2) * pl[1]) * wscale;
}

// Full weighting to the coarse grid (side nc, fine side 2nc+1): coarse point
// I sits on fine point 2I+1 (0-based); weights (1/4, 1/2, 1/4) per axis.  The
// input is the fine scaled residual r' = r/d_f and the output the coarse scaled
// right-hand side beta_c = FW(r)/d_c, so the final factor is
// wscale = d_f / (2^(2 DIM) d_c).
template <typename T, int DIM, bool RED_ONLY = false>
__global__ void __launch_bounds__(kBX* kBY)
    k_restrict(int nc, T wscale, const T* __restrict__ r, T* __restrict__ bc) {
  grid_dep_wait();
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  bc[lin<DIM>(I, J, K, nc)] = restrict_point<T, DIM, RED_ONLY>(nc, wscale, r, I, J, K);
}

// x += P e_c on the fine points of coarse cell (I,J,K): (bi/tri)linear
// interpolation from the coarse grid (side nc) to the fine grid (side
// n = 2nc+1); coarse ghosts are zero.  Cell (I,J,K) in [0, nc]^DIM owns the
// fine points {2I, 2I+1} x {2J, 2J+1} (x {2K, 2K+1}): the odd index coincides
// with coarse I, the even one lies between coarse I-1 and I.  The
// interpolated values are built from shared partial sums (2.5 operations per
// fine point in 3D).
// BLACK_ONLY: the next operation on this level is a red half sweep, which
// overwrites every red point without reading it, so only the black fine points
// (1-based index sum odd) are corrected; the result is the same.
template <typename T, int DIM, bool BLACK_ONLY>
__device__ __forceinline__ void prolong_cell(int nc, const T* __restrict__ ec, T* __restrict__ x, int I, int J,
                                             int K) {
  const int n = 2 * nc + 1;
  const bool hi_i = I > 0, ok_i = I < nc, hi_j = J > 0, ok_j = J < nc;
  const int fi = 2 * I, fj = 2 * J;
  if (DIM == 2) {
    // c_ji: j, i in {0: index-1, 1: index}
    const T c00 = (hi_i && hi_j) ? ec[(I - 1) + nc * (J - 1)] : T(0);
    const T c01 = (ok_i && hi_j) ? ec[I + nc * (J - 1)] : T(0);
    const T c10 = (hi_i && ok_j) ? ec[(I - 1) + nc * J] : T(0);
    const T c11 = (ok_i && ok_j) ? ec[I + nc * J] : T(0);
    const T sx0 = c00 + c01, sx1 = c10 + c11, sy1 = c01 + c11;
    T* xe = x + (fi + n * fj);  // (even, even); 2D fine points with ex+ey even are red
    if (!BLACK_ONLY) xe[0] = fma(T(0.25), sx0 + sx1, xe[0]);
    if (ok_i) xe[1] = fma(T(0.5), sy1, xe[1]);
    if (ok_j) {
      xe[n] = fma(T(0.5), sx1, xe[n]);
      if (ok_i && !BLACK_ONLY) xe[n + 1] += c11;
    }
  } else {
    const bool hi_k = K > 0, ok_k = K < nc;
    auto cv = [&](bool ok, int i, int j, int k) { return ok ? ec[i + nc * (j + nc * k)] : T(0); };
    // c_kji
    const T c000 = cv(hi_i && hi_j && hi_k, I - 1, J - 1, K - 1), c001 = cv(ok_i && hi_j && hi_k, I, J - 1, K - 1);
    const T c010 = cv(hi_i && ok_j && hi_k, I - 1, J, K - 1), c011 = cv(ok_i && ok_j && hi_k, I, J, K - 1);
    const T c100 = cv(hi_i && hi_j && ok_k, I - 1, J - 1, K), c101 = cv(ok_i && hi_j && ok_k, I, J - 1, K);
    const T c110 = cv(hi_i && ok_j && ok_k, I - 1, J, K), c111 = cv(ok_i && ok_j && ok_k, I, J, K);
    const T sx00 = c000 + c001, sx01 = c010 + c011, sx10 = c100 + c101, sx11 = c110 + c111;  // along x
    const T sy0 = c001 + c011, sy1 = c101 + c111;                                          // along y at i
    const T sz = c011 + c111;                                                              // along z at (j, i)
    const T sxy0 = sx00 + sx01, sxy1 = sx10 + sx11, sxz = sx01 + sx11, syz = sy0 + sy1;
    const T sxyz = sxy0 + sxy1;
    const int nn = n * n;
    T* xe = x + (fi + n * (fj + n * (2 * K)));  // (even, even, even)
    // 3D fine points with ex+ey+ez odd are red
    // even k plane
    xe[0] = fma(T(0.125), sxyz, xe[0]);
    if (ok_i && !BLACK_ONLY) xe[1] = fma(T(0.25), syz, xe[1]);
    if (ok_j) {
      if (!BLACK_ONLY) xe[n] = fma(T(0.25), sxz, xe[n]);
      if (ok_i) xe[n + 1] = fma(T(0.5), sz, xe[n + 1]);
    }
    if (ok_k) {  // odd k plane
      T* xo = xe + nn;
      if (!BLACK_ONLY) xo[0] = fma(T(0.25), sxy1, xo[0]);
      if (ok_i) xo[1] = fma(T(0.5), sy1, xo[1]);
      if (ok_j) {
        xo[n] = fma(T(0.5), sx11, xo[n]);
        if (ok_i && !BLACK_ONLY) xo[n + 1] += c111;
      }
    }
  }
}

template <typename T, int DIM, bool BLACK_ONLY = false>
__global__ void __launch_bounds__(kBX* kBY)
    k_prolong_add(int nc, const T* __restrict__ ec, T* __restrict__ x) {
  grid_dep_wait();
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  const int K = blockIdx.z;
  if (I > nc || J > nc) return;
  prolong_cell<T, DIM, BLACK_ONLY>(nc, ec, x, I, J, K);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP64 defect to FP32, FP32 correction added in FP64.
// ---------------------------------------------------------------------------
// Scaled defect in FP64, stored in FP32: r32 = fp32(beta - x + kappa * sum).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_defect(int n, double kappa, const double* __restrict__ x, const double* __restrict__ beta,
             float* __restrict__ r32) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  r32[p] = float(fma(kappa, nbsum<double, DIM>(x, i, j, k, n, p), beta[p]) - x[p]);
}

// beta = b / d (scaling of a caller's right-hand side).
template <typename T>
__global__ void k_scale(size_t N, T s, const T* __restrict__ b, T* __restrict__ beta) {
  grid_dep_wait();
  for (size_t p = blockIdx.x * size_t(blockDim.x) + threadIdx.x; p < N; p += size_t(gridDim.x) * blockDim.x)
    beta[p] = s * b[p];
}

template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_update(int n, double* __restrict__ x, const float* __restrict__ e32) {
  grid_dep_wait();
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= n || j >= n) return;
  const int p = lin<DIM>(i, j, k, n);
  x[p] += double(e32[p]);
}

// ---------------------------------------------------------------------------
// Colour-split layout of the fine level (FP32 V-cycles with red-black
// smoothing).  Each colour c has its own array with H = (n+1)/2 slots per
// row: point (i,j,k) of colour c = (i+j+k+DIM) & 1 (0-based, red = 0) sits in
// slot (i >> 1) + H * (j + n*k) of array c; in row (j,k) colour c starts at
// i0 = (c + j + k + DIM) & 1.  The x-neighbours of a slot-h point are slots
// h-1+i0 and h+i0 of the other colour in the same row, its y/z-neighbours
// slot h of the other colour in rows j+-1 / k+-1, so a colour pass reads only
// the other colour and its own rhs, all of it coalesced.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ int split_row(int j, int k, int n) {
  return DIM == 2 ? j : j + n * k;
}

// Neighbour sum of the colour-c point in slot h of row (j,k) (x index i = 2h + i0)
// from the other colour's array o; zero outside the interior.
template <int DIM>
__device__ __forceinline__ float split_nbsum(const float* __restrict__ o, int h, int i, int i0, int j, int k, int n,
                                             int H) {
  const size_t r = size_t(H) * split_row<DIM>(j, k, n);
  const float* row = o + r;
  const float sx = (i > 0 ? row[h - 1 + i0] : 0.f) + (i < n - 1 ? row[h + i0] : 0.f);
  const float sy = (j > 0 ? row[h - H] : 0.f) + (j < n - 1 ? row[h + H] : 0.f);
  if (DIM == 2) return sx + sy;
  const size_t hz = size_t(H) * n;
  const float sz = (k > 0 ? row[h - hz] : 0.f) + (k < n - 1 ? row[h + hz] : 0.f);
  return (sx + sy) + sz;
}

// FP64 defect of the node equation into the split FP32 arrays: one thread per
// slot pair (points 2h and 2h+1 of a row, one of each colour).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_defect_split(int n, double kappa, const double* __restrict__ x, const double* __restrict__ beta,
                   float* __restrict__ r0, float* __restrict__ r1) {
  grid_dep_wait();
  const int h = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  const int H = (n + 1) >> 1;
  if (h >= H || j >= n) return;
  const int c0 = (j + (DIM == 3 ? k : 0) + DIM) & 1;  // colour of the even point 2h
  const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
  float* even = c0 ? r1 : r0;
  float* odd = c0 ? r0 : r1;
  const int i = 2 * h;
  int p = lin<DIM>(i, j, k, n);
  even[slot] = float(fma(kappa, nbsum<double, DIM>(x, i, j, k, n, p), beta[p]) - x[p]);
  if (i + 1 < n) {
    ++p;
    odd[slot] = float(fma(kappa, nbsum<double, DIM>(x, i + 1, j, k, n, p), beta[p]) - x[p]);
  }
}

// u += e from the split arrays, in FP64.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_update_split(int n, double* __restrict__ x, const float* __restrict__ e0, const float* __restrict__ e1) {
  grid_dep_wait();
  const int h = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  const int H = (n + 1) >> 1;
  if (h >= H || j >= n) return;
  const int c0 = (j + (DIM == 3 ? k : 0) + DIM) & 1;
  const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
  const int p = lin<DIM>(2 * h, j, k, n);
  x[p] += double((c0 ? e1 : e0)[slot]);
  if (2 * h + 1 < n) x[p + 1] += double((c0 ? e0 : e1)[slot]);
}

// Red-black half sweep on the split layout: x_c = beta_c + kappa * (sum of the
// other colour's neighbours); zero_guess: x_c = beta_c.  Each thread walks
// ZB z-planes (3D; a compile-time count, so the loop unrolls and the loads of
// all its planes are in flight together: the colour arrays do not alias).
template <int DIM, int ZB>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs_split(int n, float kappa, int colour, float* __restrict__ xc, const float* __restrict__ xo,
                 const float* __restrict__ bc, int zero_guess) {
  grid_dep_wait();
  const int h = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int H = (n + 1) >> 1;
  if (j >= n) return;
  constexpr int nz = DIM == 3 ? ZB : 1;
#pragma unroll
  for (int kk = 0; kk < nz; ++kk) {
    const int k = DIM == 3 ? blockIdx.z * ZB + kk : 0;
    const int i0 = (colour + j + (DIM == 3 ? k : 0) + DIM) & 1;
    const int i = 2 * h + i0;
    if (k < (DIM == 3 ? n : 1) && i < n) {
      const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
      xc[slot] = zero_guess ? bc[slot] : fmaf(kappa, split_nbsum<DIM>(xo, h, i, i0, j, k, n, H), bc[slot]);
    }
  }
}

// The same with 4 consecutive slots per thread: 16-byte loads of the rhs and of
// the y/z neighbours and 16-byte stores (a row of H = (n+1)/2 slots is a power
// of two >= 4, so every row starts 16-byte aligned); the x neighbours are one
// 16-byte load plus one scalar.  Per lane the same FP32 operations in the same
// order as k_rbgs_split (bitwise equal).  A slot past the end of a row (odd n,
// i0 = 1) receives 0, which keeps that padding slot zero.
template <int DIM, int ZB>
__global__ void __launch_bounds__(kBX* kBY)
    k_rbgs_split4(int n, float kappa, int colour, float* __restrict__ xc, const float* __restrict__ xo,
                  const float* __restrict__ bc, int zero_guess) {
  grid_dep_wait();
  const int h = (blockIdx.x * kBX + threadIdx.x) * 4, j = blockIdx.y * kBY + threadIdx.y;
  const int H = (n + 1) >> 1;
  if (j >= n || h >= H) return;
  constexpr int nz = DIM == 3 ? ZB : 1;
#pragma unroll
  for (int kk = 0; kk < nz; ++kk) {
    const int k = DIM == 3 ? blockIdx.z * ZB + kk : 0;
    if (k >= (DIM == 3 ? n : 1)) continue;
    const int i0 = (colour + j + (DIM == 3 ? k : 0) + DIM) & 1;
    const size_t r = size_t(H) * split_row<DIM>(j, k, n);
    const float4 b4 = *reinterpret_cast<const float4*>(bc + r + h);
    float4 v;
    if (zero_guess) {
      v = b4;
    } else {
      const float* row = xo + r;
      // other-colour slots h-1+i0 .. h+3+i0 (x neighbours of the 4 lanes)
      const float4 m4 = *reinterpret_cast<const float4*>(row + h);
      float e[5];
      if (i0 == 0) {
        e[0] = h > 0 ? row[h - 1] : 0.f;
        e[1] = m4.x; e[2] = m4.y; e[3] = m4.z; e[4] = m4.w;
      } else {
        e[0] = m4.x; e[1] = m4.y; e[2] = m4.z; e[3] = m4.w;
        e[4] = h + 4 < H ? row[h + 4] : 0.f;
      }
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 yd = j > 0 ? *reinterpret_cast<const float4*>(row + h - H) : zero4;
      const float4 yu = j < n - 1 ? *reinterpret_cast<const float4*>(row + h + H) : zero4;
      float4 zd = zero4, zu = zero4;
      if (DIM == 3) {
        const size_t hz = size_t(H) * n;
        if (k > 0) zd = *reinterpret_cast<const float4*>(row + h - hz);
        if (k < n - 1) zu = *reinterpret_cast<const float4*>(row + h + hz);
      }
      const float ydv[4] = {yd.x, yd.y, yd.z, yd.w}, yuv[4] = {yu.x, yu.y, yu.z, yu.w};
      const float zdv[4] = {zd.x, zd.y, zd.z, zd.w}, zuv[4] = {zu.x, zu.y, zu.z, zu.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
      float out[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 2 * (h + q) + i0;
        const float sx = (i > 0 ? e[q] : 0.f) + (i < n - 1 ? e[q + 1] : 0.f);
        const float sy = ydv[q] + yuv[q];
        float sum = sx + sy;
        if (DIM == 3) sum = sum + (zdv[q] + zuv[q]);
        out[q] = i < n ? fmaf(kappa, sum, bv[q]) : 0.f;
      }
      v = make_float4(out[0], out[1], out[2], out[3]);
    }
    if (zero_guess && i0 == 1 && 2 * (h + 3) + 1 >= n) v.w = 0.f;  // padding slot stays zero
    *reinterpret_cast<float4*>(xc + r + h) = v;
  }
}

// ---------------------------------------------------------------------------
// Temporal blocking (3D, split layout): S/2 complete red-black sweeps in one
// pass over HBM.  A block owns a tile of kTbX slots x kTbY rows and a chunk
// of zc planes and walks z as a wavefront of S colour stages: at iteration
// `it` stage s (red for even s, black for odd s) updates plane it - s from the
// three planes of stage s-1 around it.  Stage s is computed on the tile plus
// a ring of S-1-s slots / rows (and S-1-s extra planes at each end of the
// chunk), so the last stage needs nothing from other blocks; the halo work is
// recomputed.  Only the black input and the right-hand sides are read from
// HBM (a Gauss-Seidel red update never reads the old red values) and only the
// last red and black stages are written: S/2 sweeps move 2.5 values per point
// instead of 3 per sweep.  The black result goes to a second array
// (xb_out != xb_in), because other blocks still read the old black values in
// their halos.  The global loads of iteration it+1 (black input plane it+2,
// right-hand-side planes it+1) are issued into registers before the stages of
// iteration it run, so the stages work out of shared memory only.  Every
// stage does the same FP32 operations in the same order as k_rbgs_split, so
// the result is bitwise that of S separate colour passes.
// ---------------------------------------------------------------------------
constexpr int kTbX = 32, kTbY = 16, kTbThreads = kTbX * kTbY;

template <int S>
struct TbShape {
  static constexpr int WX = kTbX + 2 * S, WY = kTbY + 2 * S, PL = WX * WY;
  static constexpr int LOADS = (PL + kTbThreads - 1) / kTbThreads;  // plane elements per thread
  // black input (3 planes), stages 0..S-2 (3 planes each), red and black rhs (4 planes each)
  static constexpr int BUF_IN = 0, BUF_STAGE = 3 * PL, BUF_BR = BUF_STAGE + 3 * (S - 1) * PL, BUF_BB = BUF_BR + 4 * PL;
  static constexpr size_t smem_bytes = size_t(BUF_BB + 4 * PL) * sizeof(float);
  // slot 1 of the kTbThreads threads covers every point of the rings 1..S-1
  static constexpr int RING_POINTS = (kTbX + 2 * (S - 1)) * (kTbY + 2 * (S - 1)) - kTbX * kTbY;
  static_assert(RING_POINTS <= kTbThreads, "rings 1..S-1 need more than one point per thread");
};

__device__ __forceinline__ int tb_zslot(int z, int S) { return (z + 3 * (S + 2)) % 3; }
__device__ __forceinline__ int tb_bslot(int z) { return (z + 1024) & 3; }

// A point of the shared-memory plane owned by a thread: for the stages, slot 0
// is tile point t and slot 1 the t-th point of the rings 1..S-1 around the
// tile, ring by ring (a stage with ring r uses slot 1 only where dist <= r, so
// the work stays spread over all threads); for the plane loads, element q of
// the whole buffer.  Everything but z is fixed for the whole pass: in plane z
// the colour-c point of the slot has x offset i0 = ((c + z + 1) & 1) ^ ypar and
// lies in the grid iff ok[i0].
struct TbSlot {
  int e;        // shared-memory index in a plane (-1: unused)
  int g;        // h + H*y: global slot offset within a plane
  int ypar;     // y & 1
  int dist;     // ring (0 = tile); larger than any ring when unused
  bool ok0, ok1;  // inside the grid with i0 = 0 / 1
};

template <int S>
__device__ __forceinline__ TbSlot tb_at(int hs, int ys, int dist, int n, int H, int h0, int y0) {
  TbSlot t;
  const int h = h0 - S + hs, y = y0 - S + ys;
  const bool inxy = h >= 0 && y >= 0 && y < n;
  t.e = ys * TbShape<S>::WX + hs;
  t.g = h + H * y;
  t.ypar = y & 1;
  t.dist = dist;
  t.ok0 = inxy && 2 * h < n;
  t.ok1 = inxy && 2 * h + 1 < n;
  return t;
}

template <int S>
__device__ __forceinline__ TbSlot tb_slot(int q, int ring, int n, int H, int h0, int y0) {
  if (ring == 0) return tb_at<S>(S + q % kTbX, S + q / kTbX, 0, n, H, h0, y0);
  for (int d = 1; d < S; ++d) {
    const int Wd = kTbX + 2 * d, Hd = kTbY + 2 * d, c = 2 * Wd + 2 * (Hd - 2);
    if (q < c) {
      if (q < Wd) return tb_at<S>(S - d + q, S - d, d, n, H, h0, y0);
      if (q < 2 * Wd) return tb_at<S>(S - d + (q - Wd), S + kTbY + d - 1, d, n, H, h0, y0);
      const int r = q - 2 * Wd;
      return tb_at<S>((r & 1) ? S + kTbX + d - 1 : S - d, S - d + 1 + (r >> 1), d, n, H, h0, y0);
    }
    q -= c;
  }
  TbSlot t = tb_at<S>(S, S, 1 << 20, n, H, h0, y0);
  t.e = -1;
  return t;
}

// Loads of one plane z of colour c (value 0 outside the grid) into registers.
template <int S>
__device__ __forceinline__ void tb_load(float (&v)[TbShape<S>::LOADS], const TbSlot (&ld)[TbShape<S>::LOADS],
                                        const float* __restrict__ a, int c, int z, int n, size_t plane, bool need) {
  need = need && z >= 0 && z < n;
  const float* az = a + plane * size_t(need ? z : 0);
  const int par = (c + z + 1) & 1;
#pragma unroll
  for (int k = 0; k < TbShape<S>::LOADS; ++k) {
    const TbSlot& t = ld[k];
    const bool ok = need && t.e >= 0 && ((par ^ t.ypar) ? t.ok1 : t.ok0);
    v[k] = ok ? az[t.g] : 0.f;
  }
}

template <int S>
__device__ __forceinline__ void tb_store(float* __restrict__ dst, const float (&v)[TbShape<S>::LOADS],
                                         const TbSlot (&ld)[TbShape<S>::LOADS]) {
#pragma unroll
  for (int k = 0; k < TbShape<S>::LOADS; ++k)
    if (ld[k].e >= 0) dst[ld[k].e] = v[k];
}

template <int S, int s>
__device__ __forceinline__ void tb_stage(float* __restrict__ sm, const TbSlot (&sl)[2], int it, int n, size_t plane,
                                         int z0, int z1, float kappa, float* __restrict__ xr_out,
                                         float* __restrict__ xb_out, bool zero_guess) {
  using Sh = TbShape<S>;
  constexpr int r = S - 1 - s;           // ring of this stage
  constexpr int c = s & 1;               // colour updated: 0 red, 1 black
  const int z = it - s;
  const bool active = z >= z0 - r && z < z1 + r && z >= 0 && z < n;
  const bool store = s >= S - 2 && z >= z0 && z < z1;  // last red / last black stage, own planes
  const int par = (c + z + 1) & 1;
  const float* src = sm + (s == 0 ? Sh::BUF_IN : Sh::BUF_STAGE + (s - 1) * 3 * Sh::PL);
  const float* om = src + tb_zslot(z - 1, S) * Sh::PL;
  const float* o0 = src + tb_zslot(z, S) * Sh::PL;
  const float* op = src + tb_zslot(z + 1, S) * Sh::PL;
  float* dst = s < S - 1 ? sm + Sh::BUF_STAGE + s * 3 * Sh::PL + tb_zslot(z, S) * Sh::PL : nullptr;
  const float* bz = sm + (c ? Sh::BUF_BB : Sh::BUF_BR) + tb_bslot(z) * Sh::PL;
  float* outz = (c ? xb_out : xr_out) + plane * size_t(store ? z : 0);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const TbSlot& t = sl[k];
    if (t.dist > r) continue;
    float v = 0.f;
    const int i0 = par ^ t.ypar;
    if (active && (i0 ? t.ok1 : t.ok0)) {
      const int e = t.e;
      const float bv = bz[e];
      if (s == 0 && zero_guess) {
        v = bv;
      } else {
        const float sx = o0[e - 1 + i0] + o0[e + i0];
        const float sy = o0[e - Sh::WX] + o0[e + Sh::WX];
        const float sz = om[e] + op[e];
        v = fmaf(kappa, (sx + sy) + sz, bv);
      }
      if (k == 0 && store) outz[t.g] = v;
    }
    if (dst) dst[t.e] = v;
  }
  __syncthreads();
}

template <int S, int s>
__device__ __forceinline__ void tb_stages(float* sm, const TbSlot (&sl)[2], int it, int n, size_t plane, int z0,
                                          int z1, float kappa, float* xr_out, float* xb_out, bool zero_guess) {
  tb_stage<S, s>(sm, sl, it, n, plane, z0, z1, kappa, xr_out, xb_out, zero_guess);
  if constexpr (s + 1 < S) tb_stages<S, s + 1>(sm, sl, it, n, plane, z0, z1, kappa, xr_out, xb_out, zero_guess);
}

template <int S>
__global__ void __launch_bounds__(kTbThreads, 2)
    k_rbgs_split_tb(int n, float kappa, const float* __restrict__ xb_in, float* __restrict__ xr_out,
                    float* __restrict__ xb_out, const float* __restrict__ br, const float* __restrict__ bb,
                    int zero_guess, int zc) {
  grid_dep_wait();
  using Sh = TbShape<S>;
  extern __shared__ float sm[];
  const int H = (n + 1) >> 1;
  const size_t plane = size_t(H) * n;
  const int h0 = blockIdx.x * kTbX, y0 = blockIdx.y * kTbY, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, n);
  const bool zg = zero_guess != 0;
  const TbSlot sl[2] = {tb_slot<S>(threadIdx.x, 0, n, H, h0, y0), tb_slot<S>(threadIdx.x, 1, n, H, h0, y0)};
  TbSlot ld[Sh::LOADS];
#pragma unroll
  for (int k = 0; k < Sh::LOADS; ++k) {
    const int q = threadIdx.x + k * kTbThreads;
    ld[k] = tb_at<S>(q % Sh::WX, q / Sh::WX, 0, n, H, h0, y0);
    if (q >= Sh::PL) ld[k].e = -1;
  }
  // iteration it stores the black input plane it+1 and the rhs planes it,
  // loaded during iteration it-1
  const int it_first = z0 - S - 1, it_last = z1 + S - 2;
  float vin[Sh::LOADS], vbr[Sh::LOADS], vbb[Sh::LOADS];
  tb_load<S>(vin, ld, xb_in, 1, it_first + 1, n, plane, !zg);
  tb_load<S>(vbr, ld, br, 0, it_first, n, plane, true);
  tb_load<S>(vbb, ld, bb, 1, it_first, n, plane, true);
  for (int it = it_first; it <= it_last; ++it) {
    if (!zg) tb_store<S>(sm + Sh::BUF_IN + tb_zslot(it + 1, S) * Sh::PL, vin, ld);
    tb_store<S>(sm + Sh::BUF_BR + tb_bslot(it) * Sh::PL, vbr, ld);
    tb_store<S>(sm + Sh::BUF_BB + tb_bslot(it) * Sh::PL, vbb, ld);
    __syncthreads();
    if (it < it_last) {
      const int zi = it + 2;
      tb_load<S>(vin, ld, xb_in, 1, zi, n, plane, !zg && zi >= z0 - S && zi < z1 + S);
      tb_load<S>(vbr, ld, br, 0, it + 1, n, plane, true);
      tb_load<S>(vbb, ld, bb, 1, it + 1, n, plane, true);
    }
    tb_stages<S, 0>(sm, sl, it, n, plane, z0, z1, kappa, xr_out, xb_out, zg);
  }
}

// Scaled residual at the red points after a complete red-black sweep (the
// black rows are satisfied), stored in a red-only array with the red slots.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_residual_red_split(int n, float kappa, const float* __restrict__ xr, const float* __restrict__ xb,
                         const float* __restrict__ br, float* __restrict__ rr) {
  grid_dep_wait();
  const int h = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  const int k = blockIdx.z;
  const int H = (n + 1) >> 1;
  const int i0 = (j + (DIM == 3 ? k : 0) + DIM) & 1;
  const int i = 2 * h + i0;
  if (i >= n || j >= n) return;
  const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
  rr[slot] = fmaf(kappa, split_nbsum<DIM>(xb, h, i, i0, j, k, n, H), br[slot]) - xr[slot];
}

// Full weighting from the red-only residual (the 13 / 5 red terms of
// restrict_point<RED_ONLY>) to the natural-layout coarse rhs.
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_restrict_red_split(int nc, float wscale, const float* __restrict__ rr, float* __restrict__ bc) {
  grid_dep_wait();
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= nc || J >= nc) return;
  const int n = 2 * nc + 1, H = (n + 1) >> 1;
  const int fi = 2 * I + 1, fj = 2 * J + 1, fk = 2 * K + 1;
  auto red = [&](int i, int j, int k) { return rr[size_t(i >> 1) + size_t(H) * split_row<DIM>(j, k, n)]; };
  float acc;
  if (DIM == 2) {
    acc = fmaf(4.f, red(fi, fj, 0), (red(fi - 1, fj - 1, 0) + red(fi + 1, fj - 1, 0)) +
                                        (red(fi - 1, fj + 1, 0) + red(fi + 1, fj + 1, 0))) * wscale;
  } else {
    const float e_xy = (red(fi - 1, fj - 1, fk) + red(fi + 1, fj - 1, fk)) + (red(fi - 1, fj + 1, fk) + red(fi + 1, fj + 1, fk));
    const float e_xz = (red(fi - 1, fj, fk - 1) + red(fi + 1, fj, fk - 1)) + (red(fi - 1, fj, fk + 1) + red(fi + 1, fj, fk + 1));
    const float e_yz = (red(fi, fj - 1, fk - 1) + red(fi, fj + 1, fk - 1)) + (red(fi, fj - 1, fk + 1) + red(fi, fj + 1, fk + 1));
    acc = fmaf(2.f, (e_xy + e_xz) + e_yz, 8.f * red(fi, fj, fk)) * wscale;
  }
  bc[lin<DIM>(I, J, K, nc)] = acc;
}

// Prolongation of the natural-layout coarse error onto the black points of the
// split fine level (a red half sweep follows and overwrites the red ones).
template <int DIM>
__global__ void __launch_bounds__(kBX* kBY)
    k_prolong_black_split(int nc, const float* __restrict__ ec, float* __restrict__ x0, float* __restrict__ x1) {
  grid_dep_wait();
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  const int K = blockIdx.z;
  if (I > nc || J > nc) return;
  const int n = 2 * nc + 1, H = (n + 1) >> 1;
  const bool hi_i = I > 0, ok_i = I < nc, hi_j = J > 0, ok_j = J < nc;
  const int fi = 2 * I, fj = 2 * J;
  // the black fine point at (fi + ex, fj + ey, fk + ez) sits in slot I of its row
  auto add = [&](int ex, int ey, int ez, float v) {
    const int j = fj + ey, k = DIM == 3 ? 2 * K + ez : 0;
    const int c = (fi + ex + j + k + DIM) & 1;
    float* a = c ? x1 : x0;
    a[size_t(I) + size_t(H) * split_row<DIM>(j, k, n)] += v;
  };
  if (DIM == 2) {
    const float c01 = (ok_i && hi_j) ? ec[I + nc * (J - 1)] : 0.f;
    const float c10 = (hi_i && ok_j) ? ec[(I - 1) + nc * J] : 0.f;
    const float c11 = (ok_i && ok_j) ? ec[I + nc * J] : 0.f;
    if (ok_i) add(1, 0, 0, 0.5f * (c01 + c11));
    if (ok_j) add(0, 1, 0, 0.5f * (c10 + c11));
  } else {
    const bool hi_k = K > 0, ok_k = K < nc;
    auto cv = [&](bool ok, int i, int j, int k) { return ok ? ec[i + nc * (j + nc * k)] : 0.f; };
    const float c000 = cv(hi_i && hi_j && hi_k, I - 1, J - 1, K - 1), c001 = cv(ok_i && hi_j && hi_k, I, J - 1, K - 1);
    const float c010 = cv(hi_i && ok_j && hi_k, I - 1, J, K - 1), c011 = cv(ok_i && ok_j && hi_k, I, J, K - 1);
    const float c100 = cv(hi_i && hi_j && ok_k, I - 1, J - 1, K), c101 = cv(ok_i && hi_j && ok_k, I, J - 1, K);
    const float c110 = cv(hi_i && ok_j && ok_k, I - 1, J, K), c111 = cv(ok_i && ok_j && ok_k, I, J, K);
    const float sx00 = c000 + c001, sx01 = c010 + c011, sx10 = c100 + c101, sx11 = c110 + c111;
    const float sy1 = c101 + c111, sz = c011 + c111;
    // black points of the cell: ex+ey+ez even
    add(0, 0, 0, 0.125f * ((sx00 + sx01) + (sx10 + sx11)));
    if (ok_i && ok_j) add(1, 1, 0, 0.5f * sz);
    if (ok_i && ok_k) add(1, 0, 1, 0.5f * sy1);
    if (ok_j && ok_k) add(0, 1, 1, 0.5f * sx11);
  }
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
  T kappa[kMaxLevels];   // c/d per level
  T rscale[kMaxLevels];  // restriction factor d_l / (2^(2 DIM) d_{l+1})
  int smoother, nu1, nu2;
  T omega;
  const T* Ainv;  // d * H^{-1} on the side-3 grid (acts on the scaled rhs), row-major
};

template <typename T, int DIM>
__device__ void bt_smooth(const BottomParams<T>& P, int l, T* x, const T* b, T* t) {
  const int n = P.side[l];
  const int Np = DIM == 2 ? n * n : n * n * n;
  const T kappa = P.kappa[l];
  if (P.smoother == 0) {
    for (int p = threadIdx.x; p < Np; p += blockDim.x) t[p] = x[p];
    __syncthreads();
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      x[p] = fma(P.omega, fma(kappa, nbsum<T, DIM>(t, i, j, k, n, p), b[p]) - t[p], t[p]);
    }
    __syncthreads();
  } else {
    for (int colour = 0; colour < 2; ++colour) {
      for (int p = threadIdx.x; p < Np; p += blockDim.x) {
        const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
        if (((i + j + k + DIM) & 1) != colour) continue;
        x[p] = fma(kappa, nbsum<T, DIM>(x, i, j, k, n, p), b[p]);
      }
      __syncthreads();
    }
  }
}

// The bottom V-cycle of one grid in one block; smem_raw holds 3 arrays per
// level (shared by k_bottom and the batched engine's per-instance bottoms).
template <typename T, int DIM>
__device__ __forceinline__ void bottom_vcycle(const BottomParams<T>& P, const T* __restrict__ b_top,
                                              T* __restrict__ x_top, int load_x, unsigned char* smem_raw) {
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
    const T kappa = P.kappa[l], rs = P.rscale[l];
    // after a complete red-black sweep only the red rows carry a residual
    const bool red_only = P.smoother == 1 && P.nu1 >= 1;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
      const int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      if (red_only && ((i + j + k + DIM) & 1)) continue;
      Tt[l][p] = fma(kappa, nbsum<T, DIM>(X[l], i, j, k, n, p), B[l][p]) - X[l][p];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Nc; q += blockDim.x) {
      const int I = q % nc, J = (q / nc) % nc, K = DIM == 3 ? q / (nc * nc) : 0;
      B[l + 1][q] = red_only ? restrict_point<T, DIM, true>(nc, rs, Tt[l], I, J, K)
                             : restrict_point<T, DIM, false>(nc, rs, Tt[l], I, J, K);
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
    const int nc = P.side[l + 1];
    // a red half sweep follows: correct the black points only
    const bool black_only = P.smoother == 1 && P.nu2 >= 1;
    const int cells = DIM == 2 ? (nc + 1) * (nc + 1) : (nc + 1) * (nc + 1) * (nc + 1);
    for (int q = threadIdx.x; q < cells; q += blockDim.x) {
      const int I = q % (nc + 1), J = (q / (nc + 1)) % (nc + 1), K = DIM == 3 ? q / ((nc + 1) * (nc + 1)) : 0;
      if (black_only) prolong_cell<T, DIM, true>(nc, X[l + 1], X[l], I, J, K);
      else prolong_cell<T, DIM, false>(nc, X[l + 1], X[l], I, J, K);
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

template <typename T, int DIM>
__global__ void __launch_bounds__(kBottomThreads)
    k_bottom(BottomParams<T> P, const T* __restrict__ b_top, T* __restrict__ x_top, int load_x) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bottom_vcycle<T, DIM>(P, b_top, x_top, load_x, smem_raw);
}

}  // namespace isdc
