// noalloc.cu -- isdc_vcycles_static: the standalone multigrid solve of
// isdc_vcycles without a context and without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory manager (which has already reserved the device memory),
// real-time loops that must not allocate, or code that must not allocate
// while other work is being captured into a CUDA graph.  For them the
// coarse-grid hierarchy, the fine-grid residual / Jacobi buffers and the dense
// inverse of the side-3 operator live in one file-scope static device array of
// ISDC_STATIC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  The caller passes x and b; nothing is allocated.
//
// The array's name in host code is only a host-side stand-in for the symbol,
// not a device address, so host code never hands it to a kernel: the first
// call on each device, with that device current, looks up the real address
// with cudaGetSymbolAddress and keeps it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/isdc.h"
#include "kernels.cuh"

#define ISDC_API extern "C" __attribute__((visibility("default")))

using namespace isdc;

namespace {

static __device__ __align__(256) unsigned char g_vcycle_scratch[ISDC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
#define STATIC_TRY(call)                  \
  do {                                    \
    if ((call) != cudaSuccess) return ISDC_ERR_CUDA; \
  } while (0)

// Once per device, with that device current: the device address of the
// static scratch, and the shared-memory limit of the bottom kernels.
isdc_status device_setup(void** addr) {
  int dev = 0;
  STATIC_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return ISDC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    STATIC_TRY(cudaGetSymbolAddress(&p, g_vcycle_scratch));
    const int smem = 227 * 1024;
    STATIC_TRY(cudaFuncSetAttribute(k_bottom<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    STATIC_TRY(cudaFuncSetAttribute(k_bottom<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  return ISDC_OK;
}

// Dense inverse of I - a L_h on the side-3 grid (h = 1/4), times d_3 (the
// bottom kernels apply it to beta = b / d_3), written by one block straight
// into the static array.  The operator is diagonalised by the sine basis:
// with s_q(i) = sqrt(1/2) sin(pi q i / 4) per axis (1-based i, q in {1,2,3},
// orthonormal), (I - a L_h)^{-1}[i][j] = sum_q prod_axes s_q(i) s_q(j) / mu_q,
// mu_q = 1 + (4a/h^2) sum_axes sin^2(pi q h / 2).  One thread per entry.
template <int DIM>
__global__ void k_side3_inverse(double a, double* __restrict__ inv) {
  constexpr int Np = DIM == 2 ? 9 : 27;
  __shared__ double S[3][3], mu[Np];
  const int t = threadIdx.x;
  const double c16 = 16.0 * a;  // a / h^2 with h = 1/4
  if (t < 9) S[t / 3][t % 3] = sqrt(0.5) * sinpi(double((t / 3 + 1) * (t % 3 + 1)) / 4.0);
  if (t < Np) {
    double sum = 0.0;
    for (int ax = 0, q = t; ax < DIM; ++ax, q /= 3) {
      const double sn = sinpi(double(q % 3 + 1) / 8.0);
      sum += sn * sn;
    }
    mu[t] = 1.0 + 4.0 * c16 * sum;
  }
  __syncthreads();
  if (t >= Np * Np) return;
  const int row = t / Np, col = t % Np;
  double acc = 0.0;
  for (int q = 0; q < Np; ++q) {
    double w = 1.0;
    for (int ax = 0, r = row, c = col, qq = q; ax < DIM; ++ax, r /= 3, c /= 3, qq /= 3)
      w *= S[r % 3][qq % 3] * S[c % 3][qq % 3];
    acc += w / mu[q];
  }
  inv[t] = acc * (1.0 + 2.0 * DIM * c16);
}

// The V-cycle's buffers carved out of the static scratch.
struct Layout {
  int nlev = 0, lb = 0;
  int side[kMaxLevels] = {};
  size_t npts[kMaxLevels] = {};
  size_t ainv = 0, beta = 0, x[kMaxLevels] = {}, b[kMaxLevels] = {}, r[kMaxLevels] = {}, t[kMaxLevels] = {};
  size_t bytes = 0, bottom_smem = 0;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

void plan(int dim, int n, bool jacobi, Layout& L) {
  int s = n, l = 0;
  for (;;) {
    L.side[l] = s;
    L.npts[l] = dim == 2 ? size_t(s) * s : size_t(s) * s * s;
    ++l;
    if (s <= 3) break;
    s = (s - 1) / 2;
  }
  L.nlev = l;
  const int threshold = dim == 2 ? 63 : 15;  // sides handled by the single-block bottom kernel
  L.lb = 0;
  while (L.side[L.lb] > threshold) ++L.lb;
  size_t off = 0;
  auto take = [&](size_t count) {
    const size_t o = off;
    off = align256(off + count * sizeof(double));
    return o;
  };
  L.ainv = take(dim == 2 ? 81 : 729);
  L.beta = take(L.npts[0]);
  for (int q = 0; q < L.nlev; ++q) {
    if (q < L.lb) {
      L.r[q] = take(L.npts[q]);
      if (jacobi) L.t[q] = take(L.npts[q]);
    }
    if (q > 0 && q <= L.lb) {
      L.x[q] = take(L.npts[q]);
      L.b[q] = take(L.npts[q]);
    }
  }
  L.bytes = off;
  size_t sm = 0;
  for (int q = L.lb; q < L.nlev; ++q) sm += 3 * L.npts[q] * sizeof(double);
  L.bottom_smem = sm;
}

struct Coef {
  double d, kappa;
};
inline Coef coef(int dim, int s, double a) {
  const double h = 1.0 / (s + 1), c = a / (h * h), d = 1.0 + 2.0 * dim * c;
  return {d, c / d};
}
inline double restrict_scale(int dim, int s, int sc, double a) {
  return coef(dim, s, a).d / (coef(dim, sc, a).d * (dim == 2 ? 16.0 : 64.0));
}

inline dim3 grid_pts(int dim, int s) { return dim3((s + kBX - 1) / kBX, (s + kBY - 1) / kBY, dim == 3 ? s : 1); }

struct Solve {
  int dim, smoother, nu1, nu2;
  double omega, a;
  cudaStream_t stream;
  unsigned char* base;
  Layout L;
  double* at(size_t off) const { return reinterpret_cast<double*>(base + off); }
};

template <int DIM>
isdc_status smooth(const Solve& S, int l, double*& x, double* home, const double* b, bool& zero, int sweeps) {
  const int s = S.L.side[l];
  const double kappa = coef(DIM, s, S.a).kappa;
  const dim3 blk(kBX, kBY, 1);
  for (int it = 0; it < sweeps; ++it) {
    if (S.smoother == ISDC_SMOOTHER_JACOBI) {
      double* t = S.at(S.L.t[l]);
      double* out = (x == t) ? home : t;
      k_jacobi<double, DIM><<<grid_pts(DIM, s), blk, 0, S.stream>>>(s, kappa, S.omega, x, b, out, zero ? 1 : 0);
      x = out;
    } else {
      launch_rbgs<double, DIM>(S.stream, s, kappa, 0, x, b, zero, 1);
      launch_rbgs<double, DIM>(S.stream, s, kappa, 1, x, b, false, 1);
    }
    STATIC_TRY(cudaGetLastError());
    zero = false;
  }
  return ISDC_OK;
}

template <int DIM>
isdc_status one_vcycle(const Solve& S, double* x0, const double* b0) {
  const Layout& L = S.L;
  const dim3 blk(kBX, kBY, 1);
  double* xcur[kMaxLevels];
  isdc_status st;
  for (int l = 0; l < L.lb; ++l) {
    double* home = l == 0 ? x0 : S.at(L.x[l]);
    double* x = home;
    const double* b = l == 0 ? b0 : S.at(L.b[l]);
    bool zero = l > 0;  // coarse corrections start from zero
    const int s = L.side[l];
    if (S.nu1 == 0 && zero) {
      STATIC_TRY(cudaMemsetAsync(x, 0, L.npts[l] * sizeof(double), S.stream));
      zero = false;
    }
    if ((st = smooth<DIM>(S, l, x, home, b, zero, S.nu1)) != ISDC_OK) return st;
    k_residual<double, DIM><<<grid_pts(DIM, s), blk, 0, S.stream>>>(s, coef(DIM, s, S.a).kappa, x, b,
                                                                      S.at(L.r[l]));
    k_restrict<double, DIM><<<grid_pts(DIM, L.side[l + 1]), blk, 0, S.stream>>>(
        L.side[l + 1], restrict_scale(DIM, s, L.side[l + 1], S.a), S.at(L.r[l]), S.at(L.b[l + 1]));
    STATIC_TRY(cudaGetLastError());
    xcur[l] = x;
  }
  {
    BottomParams<double> P{};
    P.nlev = L.nlev - L.lb;
    for (int q = 0; q < P.nlev; ++q) {
      const int s = L.side[L.lb + q];
      P.side[q] = s;
      P.kappa[q] = coef(DIM, s, S.a).kappa;
      P.rscale[q] = q + 1 < P.nlev ? restrict_scale(DIM, s, L.side[L.lb + q + 1], S.a) : 0.0;
    }
    P.smoother = S.smoother;
    P.nu1 = S.nu1;
    P.nu2 = S.nu2;
    P.omega = S.omega;
    P.Ainv = S.at(L.ainv);
    const double* bb = L.lb == 0 ? b0 : S.at(L.b[L.lb]);
    double* xb = L.lb == 0 ? x0 : S.at(L.x[L.lb]);
    k_bottom<double, DIM><<<1, kBottomThreads, L.bottom_smem, S.stream>>>(P, bb, xb, L.lb == 0 ? 1 : 0);
    STATIC_TRY(cudaGetLastError());
    xcur[L.lb] = xb;
  }
  for (int l = L.lb - 1; l >= 0; --l) {
    double* home = l == 0 ? x0 : S.at(L.x[l]);
    double* x = xcur[l];
    k_prolong_add<double, DIM><<<grid_pts(DIM, L.side[l + 1] + 1), blk, 0, S.stream>>>(L.side[l + 1], xcur[l + 1],
                                                                                        x);
    STATIC_TRY(cudaGetLastError());
    bool zero = false;
    if ((st = smooth<DIM>(S, l, x, home, l == 0 ? b0 : S.at(L.b[l]), zero, S.nu2)) != ISDC_OK) return st;
    xcur[l] = x;
  }
  if (xcur[0] != x0)
    STATIC_TRY(cudaMemcpyAsync(x0, xcur[0], L.npts[0] * sizeof(double), cudaMemcpyDeviceToDevice, S.stream));
  return ISDC_OK;
}

}  // namespace

ISDC_API isdc_status isdc_vcycles_static(int ndim, int64_t n, double a, int smoother, int nu1, int nu2,
                                         double omega, double* x, const double* b, int n_cycles, void* stream) {
  if (ndim != 2 && ndim != 3) return ISDC_ERR_INVALID_ARG;
  if (n < 3 || ((n + 1) & n) != 0 || n > 46339) return ISDC_ERR_INVALID_ARG;
  if (!x || !b || !(a > 0) || !std::isfinite(a) || n_cycles < 0) return ISDC_ERR_INVALID_ARG;
  if (smoother != ISDC_SMOOTHER_JACOBI && smoother != ISDC_SMOOTHER_RBGS) return ISDC_ERR_INVALID_ARG;
  if (nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || nu1 > 16 || nu2 > 16) return ISDC_ERR_INVALID_ARG;
  if (smoother == ISDC_SMOOTHER_JACOBI && !(omega > 0 && omega <= 1)) return ISDC_ERR_INVALID_ARG;
  // every level of a grid that fits the array has a slot in Layout; sides with
  // more levels than Layout holds are far beyond the array anyway
  int nlev = 1;
  for (int64_t s = n; s > 3; s = (s - 1) / 2) ++nlev;
  if (nlev > kMaxLevels || (ndim == 3 && n > 1289)) return ISDC_ERR_SCRATCH_TOO_SMALL;
  Solve S{};
  plan(ndim, int(n), smoother == ISDC_SMOOTHER_JACOBI, S.L);
  if (S.L.bytes > ISDC_STATIC_SCRATCH_BYTES) return ISDC_ERR_SCRATCH_TOO_SMALL;
  void* addr = nullptr;
  isdc_status st = device_setup(&addr);
  if (st != ISDC_OK) return st;
  S.dim = ndim;
  S.smoother = smoother;
  S.nu1 = nu1;
  S.nu2 = nu2;
  S.omega = omega;
  S.a = a;
  S.stream = static_cast<cudaStream_t>(stream);
  S.base = static_cast<unsigned char*>(addr);
  if (ndim == 2) k_side3_inverse<2><<<1, 81, 0, S.stream>>>(a, S.at(S.L.ainv));
  else k_side3_inverse<3><<<1, 729, 0, S.stream>>>(a, S.at(S.L.ainv));
  STATIC_TRY(cudaGetLastError());
  // the V-cycles act on the row-scaled system x - kappa * (neighbour sum) = b / d
  double* beta = S.at(S.L.beta);
  k_scale<double><<<4 * 152, 256, 0, S.stream>>>(S.L.npts[0], 1.0 / coef(ndim, int(n), a).d, b, beta);
  STATIC_TRY(cudaGetLastError());
  for (int c = 0; c < n_cycles; ++c) {
    st = ndim == 2 ? one_vcycle<2>(S, x, beta) : one_vcycle<3>(S, x, beta);
    if (st != ISDC_OK) return st;
  }
  return ISDC_OK;
}
