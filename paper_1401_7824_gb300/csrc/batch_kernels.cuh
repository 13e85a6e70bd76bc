// batch_kernels.cuh -- work-list kernels of the batched ISDC engine.
//
// Many independent instances (each its own grid side n, nu, M, dt) are swept
// together: every phase of an SDC sweep is one persistent, grid-stride launch
// over a work list of (instance, tile) pairs that spans all instances taking
// part in that phase.  Node state and the SDC update are FP64; the V-cycles
// run in FP32 on the error equation (defect correction, as in isdc.cu).
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

// Colour grid: q indexes (ih, j, k) with ih in [0, (n+1)/2).
template <int DIM>
__device__ __forceinline__ bool decode_colour(int q, int n, int colour, int& i, int& j, int& k) {
  const int H = (n + 1) >> 1;
  const int ih = q % H;
  const int r = q / H;
  if (DIM == 2) { j = r; k = 0; } else { j = r % n; k = r / n; }
  i = 2 * ih + ((colour + j + (DIM == 3 ? k : 0) + DIM) & 1);
  return i < n && j < n && k < (DIM == 3 ? n : 1);
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
__global__ void kb_spread(const Inst* __restrict__ insts, const List* __restrict__ list, int reaction) {
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
__global__ void kb_rhs(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int reaction) {
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
__global__ void kb_update(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int from_t) {
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n;
    if (q >= npts<DIM>(n)) continue;
    double* x = I.U + (m + 1) * size_t(npts<DIM>(n));
    x[q] += double(from_t ? I.lev[0].t[q] : I.lev[0].x[q]);
  BATCH_END
}

// End of a sweep: f_{M-1}, the max-norm SDC residual (Sec. 3) into
// rbits[instance] and the next sweep's C'_m.
template <int DIM>
__global__ void kb_sweep_end(const Inst* __restrict__ insts, const List* __restrict__ list, int reaction,
                             unsigned long long* __restrict__ rbits) {
  const List& L = *list;
  BATCH_LOOP(L)
    const int n = I.n, M = I.M;
    unsigned long long rb = 0;
    if (q < npts<DIM>(n)) {
      int i, j, k;
      decode<DIM>(q, n, i, j, k);
      const size_t N = size_t(npts<DIM>(n));
      double u[kMaxM], f[kMaxM], fe[kMaxM], qf[kMaxM];
#pragma unroll
      for (int mm = 0; mm < kMaxM; ++mm)
        if (mm < M) {
          u[mm] = I.U[mm * N + q];
          fe[mm] = reaction_term(reaction, u[mm]);
        }
      const double* ul = I.U + size_t(M - 1) * N;
      const double flast = fma(I.nu_h2, fma(-double(2 * DIM), ul[q], nbsum<double, DIM>(ul, i, j, k, n, q)),
                               reaction_term(reaction, ul[q]));
      I.F[size_t(M - 1) * N + q] = flast;
#pragma unroll
      for (int mm = 0; mm < kMaxM; ++mm) {
        if (mm < M - 1) f[mm] = I.F[mm * N + q];
        else if (mm == M - 1) f[mm] = flast;
      }
#pragma unroll
      for (int mm = 1; mm < kMaxM; ++mm)
        if (mm < M) {
          double acc = I.dtQ[mm][0] * f[0];
#pragma unroll
          for (int jj = 1; jj < kMaxM; ++jj)
            if (jj < M) acc = fma(I.dtQ[mm][jj], f[jj], acc);
          qf[mm] = acc;
          const unsigned long long bits =
              (unsigned long long)__double_as_longlong((u[0] - u[mm]) + acc) & 0x7fffffffffffffffull;
          rb = bits > rb ? bits : rb;
        }
#pragma unroll
      for (int mm = 0; mm < kMaxM - 1; ++mm)
        if (mm < M - 1) {
          const double sf = mm == 0 ? qf[1] : qf[mm + 1] - qf[mm];
          I.C[mm * N + q] = fma(-I.dtm[mm], fe[mm], sf) - u[mm + 1];
        }
    }
    // all threads of the block work on the same instance: block max, one atomic
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

template <int DIM>
__global__ void kb_rbgs(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, int colour,
                        int zero) {
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& V = I.lev[l];
    int i, j, k;
    if (!decode_colour<DIM>(q, V.n, colour, i, j, k)) continue;
    const int p = lin<DIM>(i, j, k, V.n);
    V.x[p] = zero ? V.b[p] : fmaf(I.kappa[m][l], nbsum<float, DIM>(V.x, i, j, k, V.n, p), V.b[p]);
  BATCH_END
}

// Scaled residual of level l (red points only after a red-black sweep).
template <int DIM, bool RED_ONLY>
__global__ void kb_residual(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l, int src_t) {
  const List& L = *list;
  BATCH_LOOP(L)
    const Level& V = I.lev[l];
    int i, j, k;
    if (RED_ONLY) {
      if (!decode_colour<DIM>(q, V.n, 0, i, j, k)) continue;
    } else {
      if (q >= npts<DIM>(V.n)) continue;
      decode<DIM>(q, V.n, i, j, k);
    }
    const float* x = src_t ? V.t : V.x;
    const int p = lin<DIM>(i, j, k, V.n);
    V.r[p] = fmaf(I.kappa[m][l], nbsum<float, DIM>(x, i, j, k, V.n, p), V.b[p]) - x[p];
  BATCH_END
}

template <int DIM, bool RED_ONLY>
__global__ void kb_restrict(const Inst* __restrict__ insts, const List* __restrict__ list, int m, int l) {
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

#undef BATCH_LOOP
#undef BATCH_END

}  // namespace batch
}  // namespace isdc
