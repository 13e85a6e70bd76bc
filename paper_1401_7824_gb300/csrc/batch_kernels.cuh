// batch_kernels.cuh -- work-list kernels of the batched ISDC engine.
//
// Many independent instances (each its own grid side n, nu, M, dt) are swept
// together: every phase of an SDC sweep is one persistent, grid-stride launch
// over a work list of (instance, tile) pairs that spans all instances taking
// part in that phase.  A tile is a run of points (one per thread), a 2D tile
// of coarse points (the fused damped-Jacobi passes) or a few grid rows (the
// red-black passes, one row per warp).  Node state and the SDC update are
// FP64; the V-cycles run in FP32 on the error equation (defect correction, as
// in isdc.cu).
#pragma once
#include "sdc_kernels.cuh"

namespace isdc {
namespace batch {

constexpr int kMaxInst = 256;

struct Level {
  float* x;  // unknown (the error e on level 0)
  float* t;  // Jacobi ping-pong partner
  float* b;  // scaled right-hand side
  float* r;  // scaled residual
  int n;
};

// Everything a kernel needs about one instance (device-resident table).
struct Inst {
  int n, M, nlev;
  int lb;                             // first level handled by the per-instance bottom block
  double nu_h2;                       // nu / h^2 on the fine grid
  double* U;                          // M node arrays (node-major)
  double* F;                          // f(u_m), M arrays
  double* C;                          // sweep constants C'_m (defect form), M-1 arrays
  Level lev[kMaxLevels];
  double dtm[kMaxM];                  // dt (tau_{m+1} - tau_m)
  double dtQ[kMaxM][kMaxM];           // dt * Q
  double inv_d0[kMaxM];               // fine-grid row scaling 1/d per node solve
  float kappa[kMaxM][kMaxLevels];     // per node solve and level
  float wscale[kMaxM][kMaxLevels];    // restriction factor level l -> l+1
  float* ainv;                        // per node solve: d * H^{-1} on the side-3 grid
};

// Instances taking part in one phase, with the prefix sum of their tile counts.
struct List {
  int count;
  int total;                 // tiles over all listed instances
  int inst[kMaxInst];
  int start[kMaxInst + 1];
};

// Instance of tile g (binary search over the prefix sums).
__device__ __forceinline__ int find_entry(const List& L, int g) {
  int lo = 0, hi = L.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.start[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int DIM>
__device__ __forceinline__ void decode(int q, int n, int& i, int& j, int& k) {
  i = q % n;
  const int r = q / n;
  if (DIM == 2) { j = r; k = 0; } else { j = r % n; k = r / n; }
}

template <int DIM>
__device__ __forceinline__ int npts(int n) { return DIM == 2 ? n * n : n * n * n; }

#define BATCH_LOOP(L)                                                          \
  for (int g = blockIdx.x; g < (L).total; g += gridDim.x) {                    \
    const int e_ = find_entry((L), g);                                         \
    const Inst& I = insts[(L).inst[e_]];                                       \
    const int q = (g - (L).start[e_]) * blockDim.x + threadIdx.x;

#define BATCH_END }

// ---------------------------------------------------------------------------
// FP64 SDC phases
// ---------------------------------------------------------------------------

// Start of a step: u = u_{M-1} of the previous step (or the admitted initial
// value), spread to every node; f_m = f(u).  u_{M-1} itself is only read.
template <int DIM>
__device__ __forceinline__ void pb_spread(const Inst* __restrict__ insts, const List* __restrict__ list, int reaction) {
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n;
    if (q >= npts<DIM>(n)) continue;
    int i, j, k;
    decode<DIM>(q, n, i, j, k);
    const size_t N = size_t(npts<DIM>(n));
    const double* ul = I.U + size_t(I.M - 1) * N;
    const double up = ul[q];
    const double f = reaction_term(reaction, up) +
                     I.nu_h2 * fma(-double(2 * DIM), up, nbsum<double, DIM>(ul, i, j, k, n, q));
    for (int m = 0; m < I.M; ++m) {
      if (m < I.M - 1) I.U[m * N + q] = up;
      I.F[m * N + q] = f;
    }
  BATCH_END
}

// FP64 defect of node m+1's equation at its initial guess u_{m+1}^k, scaled
// by 1/d and stored in FP32 on level 0, and f_m = f(u_m) for m >= 1 (Eq. 4).
// With C'_m = dt sum_j s_{m,j} f(u_j^k) - dt_m f^E(u_m^k) - u_{m+1}^k the
// implicit terms of b and of (I - a L_h) u_{m+1}^k cancel:
//   r = u_m^{k+1} + dt_m f^E(u_m^{k+1}) + C'_m.
template <int DIM>
__device__ __forceinline__ void pb_rhs(const Inst* __restrict__ insts, const List* __restrict__ list, int m,
                                       int reaction) {
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n;
    if (q >= npts<DIM>(n)) continue;
    int i, j, k;
    decode<DIM>(q, n, i, j, k);
    const size_t N = size_t(npts<DIM>(n));
    const double* Um = I.U + m * N;
    const double up = Um[q];
    const double fe = reaction_term(reaction, up);
    I.lev[0].b[q] = float((fma(I.dtm[m], fe, up) + I.C[m * N + q]) * I.inv_d0[m]);
    if (m >= 1)
      I.F[m * N + q] = fma(I.nu_h2, fma(-double(2 * DIM), up, nbsum<double, DIM>(Um, i, j, k, n, q)), fe);
  BATCH_END
}

// u_{m+1} += e (FP32 correction from level 0, in x or in t).
template <int DIM>
__device__ __forceinline__ void pb_update(const Inst* __restrict__ insts, const List* __restrict__ list, int m,
                                          int from_t) {
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n;
    if (q >= npts<DIM>(n)) continue;
    double* x = I.U + (m + 1) * size_t(npts<DIM>(n));
    x[q] += double(from_t ? I.lev[0].t[q] : I.lev[0].x[q]);
  BATCH_END
}

// End of a sweep: f_{M-1}, the max-norm SDC residual (Sec. 3) into
// rbits[instance] and the next sweep's C'_m, for the listed instances with M
// nodes (one list and one compiled kernel per node count).
template <int DIM, int M>
__device__ __forceinline__ void pb_sweep_end(const Inst* __restrict__ insts, const List* __restrict__ list,
                                             int reaction, unsigned long long* __restrict__ rbits) {
  static_assert(M >= 2 && M <= kMaxM, "node count out of range");
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n;
    unsigned long long rb = 0;
    if (q < npts<DIM>(n)) {
      int i, j, k;
      decode<DIM>(q, n, i, j, k);
      const size_t N = size_t(npts<DIM>(n));
      double u[M], f[M], qf[M];
#pragma unroll
      for (int mm = 0; mm < M; ++mm) u[mm] = I.U[mm * N + q];
#pragma unroll
      for (int mm = 0; mm < M - 1; ++mm) f[mm] = I.F[mm * N + q];
      const double* ul = I.U + size_t(M - 1) * N;
      const double flast = fma(I.nu_h2, fma(-double(2 * DIM), u[M - 1], nbsum<double, DIM>(ul, i, j, k, n, q)),
                               reaction_term(reaction, u[M - 1]));
      I.F[size_t(M - 1) * N + q] = flast;
      f[M - 1] = flast;
#pragma unroll
      for (int mm = 1; mm < M; ++mm) {
        double acc = I.dtQ[mm][0] * f[0];
#pragma unroll
        for (int jj = 1; jj < M; ++jj) acc = fma(I.dtQ[mm][jj], f[jj], acc);
        qf[mm] = acc;
        const unsigned long long bits =
            (unsigned long long)__double_as_longlong((u[0] - u[mm]) + acc) & 0x7fffffffffffffffull;
        rb = bits > rb ? bits : rb;
      }
#pragma unroll
      for (int mm = 0; mm < M - 1; ++mm) {
        const double sf = mm == 0 ? qf[1] : qf[mm + 1] - qf[mm];
        I.C[mm * N + q] = fma(-I.dtm[mm], reaction_term(reaction, u[mm]), sf) - u[mm + 1];
      }
    }
    // all threads of the block work on the same instance: warp max, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, rb, o);
      rb = w > rb ? w : rb;
    }
    if ((threadIdx.x & 31) == 0 && rb) atomicMax(&rbits[L.inst[e_]], rb);
  BATCH_END
}

// ---------------------------------------------------------------------------
// FP32 V-cycle phases on level l of every listed instance (solve of node m+1)
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void kb_jacobi(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, float omega,
                          int src_t, int zero) {
  grid_dep_wait();
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& V = I.lev[l];
    const int n = V.n;
    if (q >= npts<DIM>(n)) continue;
    float* dst = src_t ? V.x : V.t;
    if (zero) {
      dst[q] = omega * V.b[q];
      continue;
    }
    const float* src = src_t ? V.t : V.x;
    int i, j, k;
    decode<DIM>(q, n, i, j, k);
    const float xp = src[q];
    dst[q] = fmaf(omega, fmaf(I.kappa[m][l], nbsum<float, DIM>(src, i, j, k, n, q), V.b[q]) - xp, xp);
  BATCH_END
}

// Scaled residual of level l at every point (damped-Jacobi V-cycles).
template <int DIM>
__global__ void kb_residual(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, int src_t) {
  grid_dep_wait();
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& V = I.lev[l];
    if (q >= npts<DIM>(V.n)) continue;
    int i, j, k;
    decode<DIM>(q, V.n, i, j, k);
    const float* x = src_t ? V.t : V.x;
    V.r[q] = fmaf(I.kappa[m][l], nbsum<float, DIM>(x, i, j, k, V.n, q), V.b[q]) - x[q];
  BATCH_END
}

// ---------------------------------------------------------------------------
// Row-structured work lists (red-black Gauss-Seidel V-cycles).  A row is a
// fixed (j, k) of a grid of side s; there are s (2D) or s^2 (3D) of them.
// Tile t of an instance covers rows [t NW, t NW + NW) (NW = warps per block):
// warp w takes row t NW + w and its lanes walk the row's points.  The row's
// (j, k), base address and j/k validity are formed once per row, so the
// per-point work is the stencil itself.
// ---------------------------------------------------------------------------
// Every launch shape holds 2048 threads per SM (threads x blocks per SM), so
// the row kernels are held to 32 registers: one wave of blocks is resident and
// the grid-stride loop has no tail wave.
constexpr int kRowsMaxThreads = 512, kRowsMinBlocks = 4;

template <int DIM, class SideOf, class Body>
__device__ __forceinline__ void for_list_rows(const Inst* __restrict__ insts, const List& L, const SideOf& side_of,
                                              const Body& body) {
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int g = blockIdx.x; g < L.total; g += gridDim.x) {
    const int e = find_entry(L, g);
    const Inst& I = insts[L.inst[e]];
    const int s = side_of(I);
    const int r = (g - L.start[e]) * nw + warp;
    if (r >= (DIM == 2 ? s : s * s)) continue;
    body(I, s, DIM == 2 ? r : r % s, DIM == 2 ? 0 : r / s, lane);
  }
}

// nbsum of point i of the row starting at xr (same terms, same order).
template <int DIM>
__device__ __forceinline__ float row_nbsum(const float* __restrict__ xr, int i, int n, bool jlo, bool jhi, bool klo,
                                           bool khi) {
  const float sx = (i > 0 ? xr[i - 1] : 0.f) + (i < n - 1 ? xr[i + 1] : 0.f);
  const float sy = (jlo ? xr[i - n] : 0.f) + (jhi ? xr[i + n] : 0.f);
  if (DIM == 3) {
    const int sz = n * n;
    const float szv = (klo ? xr[i - sz] : 0.f) + (khi ? xr[i + sz] : 0.f);
    return (sx + sy) + szv;
  }
  return sx + sy;
}

// One colour of a Gauss-Seidel sweep of level l: points i of row (j, k) with
// i = j + k + DIM + colour (mod 2), x = kappa * sum + b (b on zero guesses).
template <int DIM>
__global__ void __launch_bounds__(kRowsMaxThreads, kRowsMinBlocks) kb_rbgs_rows(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l,
                             int colour, int zero) {
  grid_dep_wait();
  for_list_rows<DIM>(insts, *list, [l](const Inst& I) { return I.lev[l].n; },
                     [&](const Inst& I, int n, int j, int k, int lane) {
                       const Level& V = I.lev[l];
                       const int base = lin<DIM>(0, j, k, n);
                       float* xr = V.x + base;
                       const float* br = V.b + base;
                       const int i0 = 2 * lane + ((colour + j + k + DIM) & 1);
                       if (zero) {
                         for (int i = i0; i < n; i += 64) xr[i] = br[i];
                         return;
                       }
                       const float kap = I.kappa[m][l];
                       const bool jlo = j > 0, jhi = j < n - 1, klo = k > 0, khi = k < n - 1;
                       // two points per iteration, both loaded before either is stored
                       // (same colour: the stores alias none of the loads)
#pragma unroll 1
                       for (int i = i0; i < n; i += 128) {
                         const bool two = i + 64 < n;
                         const float s1 = row_nbsum<DIM>(xr, i, n, jlo, jhi, klo, khi), b1 = br[i];
                         float s2 = 0.f, b2 = 0.f;
                         if (two) {
                           s2 = row_nbsum<DIM>(xr, i + 64, n, jlo, jhi, klo, khi);
                           b2 = br[i + 64];
                         }
                         xr[i] = fmaf(kap, s1, b1);
                         if (two) xr[i + 64] = fmaf(kap, s2, b2);
                       }
                     });
}

// Scaled residual of level l at its red points (after a red-black sweep the
// black residual is zero).
template <int DIM>
__global__ void __launch_bounds__(kRowsMaxThreads, kRowsMinBlocks) kb_residual_red_rows(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l) {
  grid_dep_wait();
  for_list_rows<DIM>(insts, *list, [l](const Inst& I) { return I.lev[l].n; },
                     [&](const Inst& I, int n, int j, int k, int lane) {
                       const Level& V = I.lev[l];
                       const int base = lin<DIM>(0, j, k, n);
                       const float* xr = V.x + base;
                       const float* br = V.b + base;
                       float* rr = V.r + base;
                       const float kap = I.kappa[m][l];
                       const bool jlo = j > 0, jhi = j < n - 1, klo = k > 0, khi = k < n - 1;
                       // point pairs (2q, 2q + 1): the red one gets its residual, the
                       // black one 0 (never read by the red-only restriction), so every
                       // sector of r is written whole and none is read back from DRAM
                       const int par = (j + k + DIM) & 1;
#pragma unroll 1
                       for (int q = lane; 2 * q < n; q += 64) {
                         const int i = 2 * q + par, ib = 2 * q + 1 - par;
                         const bool red1 = i < n, two = 2 * q + 64 < n, red2 = i + 64 < n;
                         float s1 = 0.f, b1 = 0.f, x1 = 0.f, s2 = 0.f, b2 = 0.f, x2 = 0.f;
                         if (red1) {
                           s1 = row_nbsum<DIM>(xr, i, n, jlo, jhi, klo, khi);
                           b1 = br[i];
                           x1 = xr[i];
                         }
                         if (red2) {
                           s2 = row_nbsum<DIM>(xr, i + 64, n, jlo, jhi, klo, khi);
                           b2 = br[i + 64];
                           x2 = xr[i + 64];
                         }
                         if (red1) rr[i] = fmaf(kap, s1, b1) - x1;
                         if (ib < n) rr[ib] = 0.f;
                         if (red2) rr[i + 64] = fmaf(kap, s2, b2) - x2;
                         if (two && ib + 64 < n) rr[ib + 64] = 0.f;
                       }
                     });
}

// Full weighting of level l's red residual to b_{l+1}, one coarse row per warp.
template <int DIM>
__global__ void __launch_bounds__(kRowsMaxThreads, kRowsMinBlocks) kb_restrict_red_rows(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l) {
  grid_dep_wait();
  for_list_rows<DIM>(insts, *list, [l](const Inst& I) { return I.lev[l + 1].n; },
                     [&](const Inst& I, int nc, int cj, int ck, int lane) {
                       float* bc = I.lev[l + 1].b + lin<DIM>(0, cj, ck, nc);
                       const float w = I.wscale[m][l];
                       for (int ci = lane; ci < nc; ci += 32)
                         bc[ci] = restrict_point<float, DIM, true>(nc, w, I.lev[l].r, ci, cj, ck);
                     });
}

// x_l += P x_{l+1}, one row of coarse cells (side nc + 1) per warp; BLACK_ONLY
// when a red half sweep follows and overwrites the red points.
template <int DIM, bool BLACK_ONLY>
__global__ void __launch_bounds__(kRowsMaxThreads, kRowsMinBlocks) kb_prolong_rows(const Inst* __restrict__ insts, const List* __restrict__ list, int l) {
  grid_dep_wait();
  for_list_rows<DIM>(insts, *list, [l](const Inst& I) { return I.lev[l + 1].n + 1; },
                     [&](const Inst& I, int ncell, int cj, int ck, int lane) {
                       const int nc = ncell - 1;
                       for (int ci = lane; ci < ncell; ci += 32)
                         prolong_cell<float, DIM, BLACK_ONLY>(nc, I.lev[l + 1].x, I.lev[l].x, ci, cj, ck);
                     });
}

template <int DIM, bool RED_ONLY>
__global__ void kb_restrict(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l) {
  grid_dep_wait();
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& C = I.lev[l + 1];
    const int nc = C.n;
    if (q >= npts<DIM>(nc)) continue;
    int ci, cj, ck;
    decode<DIM>(q, nc, ci, cj, ck);
    C.b[q] = restrict_point<float, DIM, RED_ONLY>(nc, I.wscale[m][l], I.lev[l].r, ci, cj, ck);
  BATCH_END
}

template <int DIM, bool BLACK_ONLY>
__global__ void kb_prolong(const Inst* __restrict__ insts, const List* __restrict__ list, int l, int dst_t,
                           int src_t) {
  grid_dep_wait();
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& C = I.lev[l + 1];
    const int nc = C.n, ncell = nc + 1;
    if (q >= (DIM == 2 ? ncell * ncell : ncell * ncell * ncell)) continue;
    const int ci = q % ncell, r = q / ncell;
    const int cj = DIM == 2 ? r : r % ncell, ck = DIM == 2 ? 0 : r / ncell;
    prolong_cell<float, DIM, BLACK_ONLY>(nc, src_t ? C.t : C.x, dst_t ? I.lev[l].t : I.lev[l].x, ci, cj, ck);
  BATCH_END
}

// Exact solve on each instance's coarsest (side-3) grid: x = (d H^{-1}) beta.
// dst_t: write into t (where an odd number of Jacobi sweeps leaves a level's
// iterate) so that the prolongation reads one location for every instance.
template <int DIM>
__global__ void kb_coarse(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int dst_t) {
  grid_dep_wait();
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& V = I.lev[I.nlev - 1];
    const int Np = DIM == 2 ? 9 : 27;
    if (q >= Np) continue;
    const float* A = I.ainv + size_t(m) * Np * Np;
    float acc = 0.f;
    for (int c = 0; c < Np; ++c) acc = fmaf(A[q * Np + c], V.b[c], acc);
    (dst_t ? V.t : V.x)[q] = acc;
  BATCH_END
}

// ---------------------------------------------------------------------------
// Coarse levels of every listed instance in one block each: the bottom of the
// V-cycle (sides <= kBatchBottom2 in 2D, <= kBatchBottom3 in 3D) on the
// instance's own level arrays, with the single-instance path's shared-memory
// V-cycle (bottom_vcycle).  One tile = one instance; blockDim = kBottomThreads.
// ---------------------------------------------------------------------------
constexpr int kBatchBottom2 = 63, kBatchBottom3 = 15;

template <int DIM>
__device__ __forceinline__ void pb_bottom(const Inst* __restrict__ insts, const List* __restrict__ list, int m,
                                          int load_x, int smoother, int nu1, int nu2, float omega,
                                          unsigned char* smem_raw) {
  const List& L = *list;
  for (int g = blockIdx.x; g < L.total; g += gridDim.x) {
    const Inst& I = insts[L.inst[find_entry(L, g)]];
    BottomParams<float> P;
    P.nlev = I.nlev - I.lb;
    for (int q = 0; q < P.nlev; ++q) {
      P.side[q] = I.lev[I.lb + q].n;
      P.kappa[q] = I.kappa[m][I.lb + q];
      P.rscale[q] = q + 1 < P.nlev ? I.wscale[m][I.lb + q] : 0.f;
    }
    P.smoother = smoother;
    P.nu1 = nu1;
    P.nu2 = nu2;
    P.omega = omega;
    P.Ainv = I.ainv + size_t(m) * (DIM == 2 ? 81 : 729);
    const Level& V = I.lev[I.lb];
    bottom_vcycle<float, DIM>(P, V.b, V.x, load_x && I.lb == 0, smem_raw);
    __syncthreads();  // shared memory is reused by the block's next instance
  }
}

// ---------------------------------------------------------------------------
// 2D damped-Jacobi V(1, nu2 <= 1) cycles with the smoother fused into the
// transfer passes.  A tile is kFtX x TY coarse points of level l+1 and owns
// the fine points [2 I0, 2 I0 + 2 kFtX) x [2 J0, 2 J0 + 2 TY) of level l (the
// tiles of a level cover its grid, whose side is 2 nc + 1).
//   down (l): t_l = J(x_l) (one sweep, x_l = 0 on zero guesses) on the tile
//     and a ring of one, the residual of t_l on the fine points that full
//     weighting needs, b_{l+1} = FW(r) on the tile's coarse points; writes t_l
//     on the owned points and b_{l+1}: one pass over level l where the
//     separate phases make three.
//   up (l): v = t_l + P e_{l+1} on the tile and a ring of one (e_{l+1} in
//     x_{l+1}), x_l = J(v) on the owned points (nu2 = 1) or x_l = v (nu2 = 0).
// Every value is formed by the same expressions as the separate phases.
// ---------------------------------------------------------------------------
constexpr int kFtX = 32;

__device__ __forceinline__ void fused_tile_origin(int q, int nc, int ty, int& I0, int& J0) {
  const int ntx = (nc + kFtX - 1) / kFtX;
  I0 = (q % ntx) * kFtX;
  J0 = (q / ntx) * ty;
}

// Geometry of work-list tile g of level l (coarse side nc = side of level l+1).
struct FTile {
  const Inst* I;
  int n, nc, I0, J0;
};
__device__ __forceinline__ FTile fused_tile(const Inst* __restrict__ insts, const List& L, int g, int l, int ty) {
  const int e = find_entry(L, g);
  FTile t;
  t.I = &insts[L.inst[e]];
  t.n = t.I->lev[l].n;
  t.nc = t.I->lev[l + 1].n;
  fused_tile_origin(g - L.start[e], t.nc, ty, t.I0, t.J0);
  return t;
}

// Row-structured access to a tile region: warp w takes rows w, w + NW, ...
// and lane l columns l, l + 32 of each, so a row's base address and validity
// are formed once per row.  Every loop has a compile-time trip count and is
// unrolled, so a thread's loads of several rows are in flight together.
// Regions 64 or more columns wide (the fine tiles with their halos) take
// their first 64 columns this way, two full lane steps per row, and the 1..32
// columns beyond as one flattened range over the whole block, so no lane step
// covers only a few halo columns.
template <int H, int W, int NW, class Body>
__device__ __forceinline__ void for_rows(int warp, int lane, const Body& body) {
  constexpr int WM = W >= 64 ? 64 : W;  // columns walked row by row
#pragma unroll
  for (int t = 0; t < (H + NW - 1) / NW; ++t) {
    const int r = warp + NW * t;
    if (r < H) {
#pragma unroll
      for (int k = 0; k < (WM + 31) / 32; ++k) {
        const int c = lane + 32 * k;
        if (c < WM) body(r, c);
      }
    }
  }
  if constexpr (W > 64) {
    static_assert(W - 64 <= 32, "halo wider than one lane step");
    constexpr int TW = W - 64, TN = H * TW;
#pragma unroll
    for (int e0 = 0; e0 < TN; e0 += 32 * NW) {
      const int e = e0 + 32 * warp + lane;
      if (e < TN) body(e / TW, 64 + e % TW);
    }
  }
}

template <int TY>
__device__ __forceinline__ void pb_down2(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l,
                                         float omega, int zero) {
  constexpr int NW = TY;  // warps per block
  constexpr int FX = 2 * kFtX, FY = 2 * TY;
  constexpr int XW = FX + 5, XH = FY + 5;  // x on fine offsets [-2, FX + 2]
  constexpr int SW = FX + 3, SH = FY + 3;  // b and the smoothed iterate on [-1, FX + 1]
  constexpr int RW = FX + 1, RH = FY + 1;  // residual on [0, FX]
  __shared__ float sx[XH][XW], sb[SH][SW], st[SH][SW], sr[RH][RW];
  const List& L = *list;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < L.total; g += gridDim.x) {
    const FTile t = fused_tile(insts, L, g, l, TY);
    const Inst& I = *t.I;
    const int n = t.n, nc = t.nc, I0 = t.I0, J0 = t.J0, fi0 = 2 * I0, fj0 = 2 * J0;
    const float kappa = I.kappa[m][l], ws = I.wscale[m][l];
    const float* __restrict__ fx = I.lev[l].x;
    const float* __restrict__ fb = I.lev[l].b;
    float* __restrict__ gt = I.lev[l].t;
    float* __restrict__ gbc = I.lev[l + 1].b;
    const unsigned un = unsigned(n);
    if (!zero)
      for_rows<XH, XW, NW>(warp, lane, [&](int r, int c) {
        const int i = fi0 - 2 + c, j = fj0 - 2 + r;
        sx[r][c] = (unsigned(i) < un && unsigned(j) < un) ? fx[i + n * j] : 0.f;
      });
    for_rows<SH, SW, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 - 1 + c, j = fj0 - 1 + r;
      sb[r][c] = (unsigned(i) < un && unsigned(j) < un) ? fb[i + n * j] : 0.f;
    });
    __syncthreads();
    for_rows<SH, SW, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 - 1 + c, j = fj0 - 1 + r;
      float v = 0.f;
      if (unsigned(i) < un && unsigned(j) < un) {
        if (zero) {
          v = omega * sb[r][c];
        } else {
          const float xp = sx[r + 1][c + 1];
          const float nb = (sx[r + 1][c] + sx[r + 1][c + 2]) + (sx[r][c + 1] + sx[r + 2][c + 1]);
          v = fmaf(omega, fmaf(kappa, nb, sb[r][c]) - xp, xp);
        }
      }
      st[r][c] = v;
    });
    __syncthreads();
    for_rows<RH, RW, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 + c, j = fj0 + r;
      float res = 0.f;
      if (unsigned(i) < un && unsigned(j) < un) {
        const float tp = st[r + 1][c + 1];
        const float nb = (st[r + 1][c] + st[r + 1][c + 2]) + (st[r][c + 1] + st[r + 2][c + 1]);
        res = fmaf(kappa, nb, sb[r + 1][c + 1]) - tp;
        if (c < FX && r < FY) gt[i + n * j] = tp;
      }
      sr[r][c] = res;
    });
    __syncthreads();
    {  // one coarse point per thread: (I0 + lane, J0 + warp)
      const int Ic = I0 + lane, Jc = J0 + warp;
      if (Ic < nc && Jc < nc) {
        const int li = 2 * lane + 1, lj = 2 * warp + 1;
        float row[3];
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
          row[dj + 1] = (sr[lj + dj][li - 1] + sr[lj + dj][li + 1]) + 2.f * sr[lj + dj][li];
        gbc[Ic + nc * Jc] = ((row[0] + row[2]) + 2.f * row[1]) * ws;
      }
    }
    __syncthreads();  // shared memory is refilled for the block's next tile
  }
}

template <int TY>
__device__ __forceinline__ void pb_up2(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l,
                                       float omega, int nu2) {
  constexpr int NW = TY;
  constexpr int FX = 2 * kFtX, FY = 2 * TY;
  constexpr int VW = FX + 2, VH = FY + 2;     // corrected iterate on fine offsets [-1, FX]
  constexpr int EW = kFtX + 2, EH = TY + 2;   // coarse error on [I0 - 1, I0 + kFtX] x [J0 - 1, J0 + TY]
  __shared__ float sv[VH][VW], se[EH][EW];
  const List& L = *list;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < L.total; g += gridDim.x) {
    const FTile t = fused_tile(insts, L, g, l, TY);
    const Inst& I = *t.I;
    const int n = t.n, nc = t.nc, I0 = t.I0, J0 = t.J0, fi0 = 2 * I0, fj0 = 2 * J0;
    const float kappa = I.kappa[m][l];
    const float* __restrict__ ft = I.lev[l].t;
    const float* __restrict__ fb = I.lev[l].b;
    const float* __restrict__ cx = I.lev[l + 1].x;
    float* __restrict__ gx = I.lev[l].x;
    const unsigned un = unsigned(n), unc = unsigned(nc);
    for_rows<EH, EW, NW>(warp, lane, [&](int r, int c) {
      const int ci = I0 - 1 + c, cj = J0 - 1 + r;
      se[r][c] = (unsigned(ci) < unc && unsigned(cj) < unc) ? cx[ci + nc * cj] : 0.f;
    });
    for_rows<VH, VW, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 - 1 + c, j = fj0 - 1 + r;
      sv[r][c] = (unsigned(i) < un && unsigned(j) < un) ? ft[i + n * j] : 0.f;
    });
    __syncthreads();
    // + P e: coarse ci sits on fine 2 ci + 1, so an odd fine index takes one
    // coarse value and an even one the mean of its two neighbours (zero ghosts);
    // fine offset c (index fi0 - 1 + c) has its coarse neighbours at se column
    // c / 2 (and c / 2 + 1 for an even index)
    for_rows<VH, VW, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 - 1 + c, j = fj0 - 1 + r;
      if (unsigned(i) < un && unsigned(j) < un) {
        const int ex = c >> 1, ey = r >> 1;
        float pe;
        if (i & 1) pe = (j & 1) ? se[ey][ex] : 0.5f * (se[ey][ex] + se[ey + 1][ex]);
        else pe = (j & 1) ? 0.5f * (se[ey][ex] + se[ey][ex + 1])
                          : 0.25f * ((se[ey][ex] + se[ey][ex + 1]) + (se[ey + 1][ex] + se[ey + 1][ex + 1]));
        sv[r][c] += pe;
      }
    });
    __syncthreads();
    for_rows<FY, FX, NW>(warp, lane, [&](int r, int c) {
      const int i = fi0 + c, j = fj0 + r;
      if (unsigned(i) < un && unsigned(j) < un) {
        const float vp = sv[r + 1][c + 1];
        float out = vp;
        if (nu2) {
          const float nb = (sv[r + 1][c] + sv[r + 1][c + 2]) + (sv[r][c + 1] + sv[r + 2][c + 1]);
          out = fmaf(omega, fmaf(kappa, nb, fb[i + n * j]) - vp, vp);
        }
        gx[i + n * j] = out;
      }
    });
    __syncthreads();  // shared memory is refilled for the block's next tile
  }
}

// Kernels of the phases (one launch each in the tick's graph).
template <int DIM>
__global__ void kb_spread(const Inst* __restrict__ insts, const List* __restrict__ list, int reaction) {
  grid_dep_wait();
  pb_spread<DIM>(insts, list, reaction);
}
template <int DIM>
__global__ void kb_rhs(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int reaction) {
  grid_dep_wait();
  pb_rhs<DIM>(insts, list, m, reaction);
}
template <int DIM>
__global__ void kb_update(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int from_t) {
  grid_dep_wait();
  pb_update<DIM>(insts, list, m, from_t);
}
template <int DIM, int M>
__global__ void kb_sweep_end(const Inst* __restrict__ insts, const List* __restrict__ list, int reaction,
                             unsigned long long* __restrict__ rbits) {
  grid_dep_wait();
  pb_sweep_end<DIM, M>(insts, list, reaction, rbits);
}
template <int DIM>
__global__ void __launch_bounds__(kBottomThreads)
    kb_bottom(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int load_x, int smoother,
              int nu1, int nu2, float omega) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pb_bottom<DIM>(insts, list, m, load_x, smoother, nu1, nu2, omega, smem_raw);
}
template <int TY>
__global__ void __launch_bounds__(32 * TY, 64 / TY)
    kb_down2(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, float omega, int zero) {
  grid_dep_wait();
  pb_down2<TY>(insts, list, m, l, omega, zero);
}
template <int TY>
__global__ void __launch_bounds__(32 * TY, 64 / TY)
    kb_up2(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, float omega, int nu2) {
  grid_dep_wait();
  pb_up2<TY>(insts, list, m, l, omega, nu2);
}

// ---------------------------------------------------------------------------
// The whole tick as one persistent cooperative launch (fused 2D mode): the
// blocks walk the tick's phase table, and a grid barrier separates phases.
// The launch is cooperative, so every block is resident and the barrier cannot
// wait for a block that has not started; still, every wait is bounded: a block
// that waits longer than kBarrierNs sets the error flag, every block leaves at
// its next barrier, and the host reports the tick as failed.  Each phase runs
// the same device function as its graph-node kernel, so both forms give the
// same result bit for bit.
// ---------------------------------------------------------------------------
enum PhaseKind { PH_SPREAD = 0, PH_SWEEP_END = 1, PH_RHS = 2, PH_DOWN = 3, PH_BOTTOM = 4, PH_UP = 5, PH_UPDATE = 6 };

struct Phase {
  int kind, list, m, l, arg;  // arg: M (sweep end), 1 = rbits / 0 = scratch (sweep end), zero guess, load_x
  int arg2;
};

struct GridBarrier {
  unsigned int count, gen;
  int err, pad;
};

constexpr unsigned long long kBarrierNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the tick has failed (a wait ran out here or elsewhere).
// expected: the arrivals that complete the barrier (gridDim.x in the tick);
// limit_ns: how long a block waits for them before it sets the error flag.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned int expected, unsigned long long limit_ns) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* verr = &gb->err;
    const unsigned int g0 = *vgen;  // read before arriving: the generation cannot move until we arrive
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == expected - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g0 && !*verr) {
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&gb->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = *verr == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <int TY>
__global__ void __launch_bounds__(32 * TY)
    kb_tick2(const Inst* __restrict__ insts, const List* __restrict__ lists, const Phase* __restrict__ phases,
             int nphases, int reaction, float omega, int nu1, int nu2, unsigned long long* __restrict__ rbits,
             unsigned long long* __restrict__ scratch, GridBarrier* gb) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int q = 0; q < nphases; ++q) {
    const Phase P = phases[q];
    const List* L = lists + P.list;
    switch (P.kind) {
      case PH_SPREAD: pb_spread<2>(insts, L, reaction); break;
      case PH_SWEEP_END: {
        unsigned long long* out = P.arg2 ? rbits : scratch;
        switch (P.arg) {
          case 2: pb_sweep_end<2, 2>(insts, L, reaction, out); break;
          case 3: pb_sweep_end<2, 3>(insts, L, reaction, out); break;
          case 4: pb_sweep_end<2, 4>(insts, L, reaction, out); break;
          case 5: pb_sweep_end<2, 5>(insts, L, reaction, out); break;
          case 6: pb_sweep_end<2, 6>(insts, L, reaction, out); break;
          default: pb_sweep_end<2, 7>(insts, L, reaction, out); break;
        }
        break;
      }
      case PH_RHS: pb_rhs<2>(insts, L, P.m, reaction); break;
      case PH_DOWN: pb_down2<TY>(insts, L, P.m, P.l, omega, P.arg); break;
      case PH_BOTTOM: pb_bottom<2>(insts, L, P.m, P.arg, 0, nu1, nu2, omega, smem_raw); break;
      case PH_UP: pb_up2<TY>(insts, L, P.m, P.l, omega, nu2); break;
      default: pb_update<2>(insts, L, P.m, 0); break;
    }
    if (q + 1 < nphases && !grid_barrier(gb, gridDim.x, kBarrierNs)) return;
  }
}

// Self-test of the bounded barrier (cooperative launch, every block resident):
// two barrier rounds that expect `phantom` more arrivals than there are
// blocks.  With phantom = 0 both complete; otherwise every block's wait runs
// out after limit_ns, the error flag is set and every block returns.
__global__ void kb_barrier_selftest(GridBarrier* gb, unsigned int phantom, unsigned long long limit_ns) {
  for (int r = 0; r < 2; ++r)
    if (!grid_barrier(gb, gridDim.x + phantom, limit_ns)) return;
}

#undef BATCH_LOOP
#undef BATCH_END

}  // namespace batch
}  // namespace isdc
