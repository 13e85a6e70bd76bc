// resrestrict.cuh -- fused residual + full-weighting restriction: one launch
// per level in which the fine residual of the level equation never leaves the
// chip.  Multigrid is not described in the paper (Acknowledgments); the
// operation is the textbook one: r = beta - x + kappa * (neighbour sum) on the
// fine grid (the row-scaled residual (b - H x)/d), then beta_c = FW(r) * wscale
// on the coarse grid (weights (1/4, 1/2, 1/4) per axis, coarse I on fine 2I+1).
//
// A block owns a tile of kRrTX x kRrTY coarse points and (3D) a chunk of kc
// coarse planes.  It evaluates the fine residual on the tile's fine region
// (2 kRrTX + 1 points by 2 kRrTY + 1 rows per plane) into shared memory and
// walks z: coarse plane K needs fine planes 2K, 2K+1 and 2K+2, so a ring of
// three planes holds them and each step adds the two new planes (plane 2K+2
// is plane 2K of the next step).  Tile edges are evaluated by both tiles that
// touch them (about 16 % extra residual work in 3D at kc = 8); HBM sees x
// and beta once and beta_c once, where the two-kernel form also writes and
// re-reads r.
//
// RED_ONLY (after a complete red-black sweep every black row is satisfied):
// only the red points (index sum + DIM even, 0-based) carry a residual, so only
// they are evaluated, stored compactly (red point at local x offset il in slot
// il >> 1 of its row) and combined with the 13 (3D) / 5 (2D) red terms of full
// weighting.  The residual and the restriction sums are the same expressions
// in the same order as k_residual / k_restrict (and k_residual_red_split /
// k_restrict_red_split), so the result equals the two-kernel form.
#pragma once
#include "kernels.cuh"

namespace isdc {

constexpr int kRrTX = 32;  // coarse points per tile along x (one warp)
constexpr int kRrTY = 8;   // coarse rows per tile
constexpr int kRrThreads = kRrTX * kRrTY;

// Residual of the natural-layout level at fine point (i, j, k).
template <typename T, int DIM>
struct ResNatural {
  const T* __restrict__ x;
  const T* __restrict__ beta;
  T kappa;
  int n;
  __device__ __forceinline__ T operator()(int i, int j, int k) const {
    const int p = lin<DIM>(i, j, k, n);
    return fma(kappa, nbsum<T, DIM>(x, i, j, k, n, p), beta[p]) - x[p];
  }
};

// Residual at a red point of the colour-split FP32 fine level (red array xr
// with its rhs br, black array xb; H slots per row).
template <int DIM>
struct ResSplitRed {
  const float* __restrict__ xr;
  const float* __restrict__ xb;
  const float* __restrict__ br;
  float kappa;
  int n, H;
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    const int h = i >> 1, i0 = i & 1;
    const size_t slot = size_t(h) + size_t(H) * split_row<DIM>(j, k, n);
    return fmaf(kappa, split_nbsum<DIM>(xb, h, i, i0, j, k, n, H), br[slot]) - xr[slot];
  }
};

template <typename T, int DIM, bool RED_ONLY, class Src>
__device__ __forceinline__ void resrestrict_tile(const Src& src, int nc, T wscale, T* __restrict__ bc, int kc) {
  constexpr int W = RED_ONLY ? kRrTX + 1 : 2 * kRrTX + 1;  // stored entries per fine row (33 / 65)
  constexpr int R = 2 * kRrTY + 1;                        // fine rows per tile (17)
  constexpr int NPL = DIM == 3 ? 3 : 1;                   // ring of fine planes
  constexpr int kWarps = kRrThreads / 32;
  __shared__ T sr[NPL][R][W];
  const int n = 2 * nc + 1;
  const int I0 = blockIdx.x * kRrTX, J0 = blockIdx.y * kRrTY;
  const int fi0 = 2 * I0, fj0 = 2 * J0;
  const int lane = threadIdx.x, warp = threadIdx.y;

  // Residual at local column col of fine row `row` in plane z, stored in the
  // ring; a point outside the grid (or, for the red layout, past the tile's
  // last fine column 2 kRrTX) is skipped.
  auto put = [&](int z, int row, int col) {
    const int j = fj0 + row;
    const int il = RED_ONLY ? 2 * col + ((j + (DIM == 3 ? z : 0) + DIM) & 1) : col;
    const int i = fi0 + il;
    if (il <= 2 * kRrTX && i < n && j < n) sr[DIM == 3 ? z % 3 : 0][row][col] = src(i, j, z);
  };
  // Fine planes z0 .. z0 + nz - 1 (2D: the one plane z0 = 0): one job per
  // (plane, row) over its first 32 (red) or 64 (all) columns, one warp each,
  // coalesced along x (the job loop is unrolled so that each thread's loads of
  // several rows are in flight together); then the last column of every
  // (plane, row), one thread each.
  auto fill = [&](int z0, int nz) {
    const int rows = nz * R;
#pragma unroll
    for (int t = 0; t < (2 * R + kWarps - 1) / kWarps; ++t) {
      const int job = warp + kWarps * t;
      if (job < rows) {
        const int pl = job / R, row = job - pl * R;
        put(z0 + pl, row, lane);
        if (!RED_ONLY) put(z0 + pl, row, lane + 32);
      }
    }
    const int tid = lane + 32 * warp;
    if (tid < rows) {
      const int pl = tid / R, row = tid - pl * R;
      put(z0 + pl, row, W - 1);
    }
  };
  // stored residual at local fine offsets (li, lj) of ring plane pl
  auto at = [&](int pl, int lj, int li) -> T { return sr[pl][lj][RED_ONLY ? (li >> 1) : li]; };

  const int I = I0 + lane, J = J0 + warp;
  const bool mine = I < nc && J < nc;
  const int li = 2 * lane + 1, lj = 2 * warp + 1;

  if (DIM == 2) {
    fill(0, 1);
    __syncthreads();
    if (!mine) return;
    T acc;
    if (RED_ONLY) {
      acc = fma(T(4), at(0, lj, li), (at(0, lj - 1, li - 1) + at(0, lj - 1, li + 1)) +
                                         (at(0, lj + 1, li - 1) + at(0, lj + 1, li + 1))) * wscale;
    } else {
      T row[3];
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
        row[dj + 1] = (at(0, lj + dj, li - 1) + at(0, lj + dj, li + 1)) + T(2) * at(0, lj + dj, li);
      acc = ((row[0] + row[2]) + T(2) * row[1]) * wscale;
    }
    bc[lin<2>(I, J, 0, nc)] = acc;
    return;
  }

  const int K0 = blockIdx.z * kc, K1 = min(nc, K0 + kc);
  if (K0 >= K1) return;  // uniform over the block
  fill(2 * K0, 1);
  for (int K = K0; K < K1; ++K) {
    fill(2 * K + 1, 2);  // 2K + 2 <= 2 nc = n - 1: always inside
    __syncthreads();
    if (mine) {
      const int P0 = (2 * K) % 3, P1 = (2 * K + 1) % 3, P2 = (2 * K + 2) % 3;
      T acc;
      if (RED_ONLY) {
        const T e_xy = (at(P1, lj - 1, li - 1) + at(P1, lj - 1, li + 1)) + (at(P1, lj + 1, li - 1) + at(P1, lj + 1, li + 1));
        const T e_xz = (at(P0, lj, li - 1) + at(P0, lj, li + 1)) + (at(P2, lj, li - 1) + at(P2, lj, li + 1));
        const T e_yz = (at(P0, lj - 1, li) + at(P0, lj + 1, li)) + (at(P2, lj - 1, li) + at(P2, lj + 1, li));
        acc = fma(T(2), (e_xy + e_xz) + e_yz, T(8) * at(P1, lj, li)) * wscale;
      } else {
        const int Pk[3] = {P0, P1, P2};
        T pl[3];
#pragma unroll
        for (int dk = 0; dk < 3; ++dk) {
          T row[3];
#pragma unroll
          for (int dj = -1; dj <= 1; ++dj)
            row[dj + 1] = (at(Pk[dk], lj + dj, li - 1) + at(Pk[dk], lj + dj, li + 1)) + T(2) * at(Pk[dk], lj + dj, li);
          pl[dk] = (row[0] + row[2]) + T(2) * row[1];
        }
        acc = ((pl[0] + pl[2]) + T(2) * pl[1]) * wscale;
      }
      bc[lin<3>(I, J, K, nc)] = acc;
    }
    __syncthreads();  // the next step overwrites planes 2K and 2K+1
  }
}

// Natural layout (every level of the hierarchy above the bottom block).
template <typename T, int DIM, bool RED_ONLY>
__global__ void __launch_bounds__(kRrThreads)
    k_resrestrict(int nc, T kappa, T wscale, const T* __restrict__ x, const T* __restrict__ beta,
                  T* __restrict__ bc, int kc) {
  grid_dep_wait();
  const ResNatural<T, DIM> src{x, beta, kappa, 2 * nc + 1};
  resrestrict_tile<T, DIM, RED_ONLY>(src, nc, wscale, bc, kc);
}

// Colour-split FP32 fine level after a complete red-black sweep.
template <int DIM>
__global__ void __launch_bounds__(kRrThreads)
    k_resrestrict_red_split(int nc, float kappa, float wscale, const float* __restrict__ xr,
                            const float* __restrict__ xb, const float* __restrict__ br, float* __restrict__ bc,
                            int kc) {
  grid_dep_wait();
  const int n = 2 * nc + 1;
  const ResSplitRed<DIM> src{xr, xb, br, kappa, n, (n + 1) >> 1};
  resrestrict_tile<float, DIM, true>(src, nc, wscale, bc, kc);
}

// Coarse planes per block (3D) when not tuned: longer chunks amortise the
// chunk's first fine plane, shorter ones give small levels enough blocks.
inline int resrestrict_kc(int nc) { return nc >= 255 ? 16 : nc >= 127 ? 8 : 4; }

// Launch shape: tiles of kRrTX x kRrTY coarse points, chunks of kc coarse planes.
inline dim3 resrestrict_grid(int dim, int nc, int kc) {
  return dim3((nc + kRrTX - 1) / kRrTX, (nc + kRrTY - 1) / kRrTY, dim == 3 ? (nc + kc - 1) / kc : 1);
}

}  // namespace isdc
