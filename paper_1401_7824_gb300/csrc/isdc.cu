// isdc.cu -- host side of the GB300 ISDC library: collocation tables, device
// state, the V-cycle and sweep drivers, and the C ABI declared in isdc.h.
//
// One time step (Sec. 2, Eq. 4 with W = I; Sec. 3):
//   spread u to the M Gauss-Lobatto nodes, f_m = f(u_m)
//   sweep k = 1, 2, ...:
//     for m = 0..M-2: b = u_m + dt_m f^E(u_m) + C_m      (k_rhs, also stores f_m)
//                     L V-cycles on (I - dt_m nu L_h) u_{m+1} = b, from u_{m+1}^k
//     f_{M-1}, SDC residual R, next C_m                   (k_sweep_end)
//   until R < tol (or a fixed sweep count); u <- u_{M-1} (tau = 1).
// FP32 V-cycles with a fixed count form the FP32 defect of u_{m+1}^k directly
// (k_rhs_defect, sweep constants C'_m): b itself is never stored.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/isdc.h"
#include "host_util.h"
#include "kernels.cuh"
#include "sdc_kernels.cuh"
#include "compact_kernels.cuh"
#include "periodic_kernels.cuh"
#include "resrestrict.cuh"

#define ISDC_API extern "C" __attribute__((visibility("default")))

using namespace isdc;
using namespace isdc::host;

namespace {

thread_local char g_create_error[512] = "";

// ---------------------------------------------------------------------------
// Multigrid hierarchy in one precision.
// ---------------------------------------------------------------------------
template <typename T>
struct Hier {
  int nlev = 0;         // levels: sides n, (n-1)/2, ..., 3
  int lb = 0;           // first level handled by the single-block bottom kernel
  int side[kMaxLevels] = {};
  size_t npts[kMaxLevels] = {};
  T* x[kMaxLevels] = {};  // level unknown (level 0: not owned, except FP32 mode)
  T* b[kMaxLevels] = {};  // level right-hand side (level 0: not owned, except FP32 mode)
  T* t[kMaxLevels] = {};  // Jacobi ping-pong partner
  T* r[kMaxLevels] = {};  // residual before restriction
  T* Ainv = nullptr;      // dense side-3 inverses, one slot per node plus one spare
  size_t bottom_smem = 0;
};

// Kernel classes timed by the built-in profiler (isdc_profile_*).
enum ProfClass {
  PC_SPREAD, PC_EVAL_F, PC_RHS, PC_SWEEP_END, PC_SMOOTH0, PC_RESIDUAL0, PC_RESTRICT0, PC_PROLONG0,
  PC_SMOOTHC, PC_RESIDUALC, PC_RESTRICTC, PC_PROLONGC, PC_BOTTOM, PC_DEFECT, PC_UPDATE, PC_RESNORM, PC_WINV,
  PC_RESRESTRICT0, PC_RESRESTRICTC, PC_COUNT
};
const char* const kProfNames[PC_COUNT] = {
    "spread", "eval_f", "rhs", "sweep_end", "smooth_fine", "residual_fine", "restrict_fine", "prolong_fine",
    "smooth_coarse", "residual_coarse", "restrict_coarse", "prolong_coarse", "bottom", "defect", "update",
    "resnorm", "w_inverse", "resrestrict_fine", "resrestrict_coarse"};

struct Profiler {
  bool on = false;
  unsigned event_mask = 0;  // classes bracketed by CUDA events
  struct Rec { cudaEvent_t e0, e1; int cls; };
  std::vector<Rec> pool;
  size_t used = 0;
  double ms[PC_COUNT] = {}, bytes[PC_COUNT] = {}, dp_ops[PC_COUNT] = {}, sp_ops[PC_COUNT] = {};
  long long launches[PC_COUNT] = {};
  // While a sweep graph is captured, events go to gpool (they become event
  // nodes of the graph and are re-recorded on every replay) and the counts to
  // the per-sweep deltas, which are added once per replay.
  bool capturing = false;
  std::vector<Rec> gpool;
  size_t gused = 0;
  double d_bytes[PC_COUNT] = {}, d_dp[PC_COUNT] = {}, d_sp[PC_COUNT] = {};
  long long d_launches[PC_COUNT] = {};
};

}  // namespace

struct isdc_ctx {
  int dim = 0, n = 0, M = 0;
  size_t N = 0;
  double nu = 0, dt = 0, h = 0;
  isdc_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int node_kind = 0;  // isdc_node_type
  int P = 0, off = 0;  // points of a sweep (t_0 and the nodes) and P - M; node j is point j + off
  double tau[kMaxM] = {}, Q[kMaxM * kMaxM] = {}, S[kMaxM * kMaxM] = {};
  SweepTables tables{};
  EndWeights ends{};   // dt * full-step weights (Gauss-Legendre end quadrature)
  double* U = nullptr;  // P point arrays (t_0, then the nodes), point-major
  double* F = nullptr;  // f(u_p), P arrays
  double* C = nullptr;  // sweep constants, P-1 arrays
  int stencil = 0;      // 0: 5/7-point, W = I; 1: 4th-order compact with W (2D)
  double* G = nullptr;  // compact: nu L_9 u per point (P arrays); F holds f~ = W f^E + nu L_9 u
  double* Rs = nullptr; // compact: W-weighted SDC residuals and two Jacobi iterates, 3 (P-1) arrays
  int equation = 0;     // 0: reaction-diffusion, Dirichlet; 1: viscous Burgers, periodic (h = 2/n)
  double* FE = nullptr; // f^E(u_p) per point (P arrays; Burgers: the WENO5 advection); not for the compact stencil
  double* b = nullptr;  // right-hand side of the current node solve
  double* u_dev = nullptr;  // device copy of u for isdc_step_host
  Hier<double> h64;
  Hier<float> h32;
  // FP32 red-black mode: the fine level's error, defect and red residual in
  // the colour-split layout (two colour arrays of hn = (n+1)/2 * n^(dim-1))
  float* sp_x = nullptr;
  float* sp_b = nullptr;
  float* sp_r = nullptr;
  size_t hn = 0;
  unsigned long long* d_scal = nullptr;  // [0] SDC residual bits, [1] node-residual bits
  unsigned long long* h_scal = nullptr;  // pinned mirror of d_scal
  unsigned long long* h_hist = nullptr;  // pinned residual bits per sweep
  int hist_cap = 0;
  int record_history = 0;
  int last_sweeps = 0, hist_count = 0;
  long long last_vcycles = 0;
  int nodes_pending = 0;
  int cprime = 0;  // this step keeps the sweep constants in the defect form C'_m (k_rhs_defect)
  int spare_slot = 0;  // Ainv slot for isdc_vcycles
  Profiler prof;
  // one SDC sweep (fixed V-cycle count) captured as a CUDA graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t sweep_graph = nullptr;
  int graph_vcycles = 0;
  unsigned graph_mask = 0;  // profiler classes with event nodes in the graph
  bool graph_counted = false;  // captured with the profiler on (per-class launch counts recorded)
  // points per thread of the red-black smoothers (autotuned): the diagonal run
  // of k_rbgs3 on natural-layout levels, z-planes of the split FP32 level
  int zb64 = 1, zb32 = 1;
  int tb_depth = 0, tb_zc = 32;  // temporal blocking of the split FP32 fine level (sweeps per pass, planes per block)
  float* sp_xb = nullptr;        // second black array of the split level (blocked passes ping-pong into it)
  // per grid-wide level (natural layout): run length, negative for burst runs (launch_rbgs)
  int zbl[kMaxLevels] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  // residual + restriction per grid-wide level of the FP64 / FP32 hierarchy:
  // 0 two launches, > 0 one fused launch with that many coarse planes per
  // block (2D: 1); rr_split: the same for the colour-split FP32 fine level
  int rr64[kMaxLevels] = {}, rr32[kMaxLevels] = {}, rr_split = 0;
  char err[512] = "";
};

namespace {

isdc_status fail(isdc_ctx* ctx, isdc_status st, const char* fmt, ...) {
  char* dst = ctx ? ctx->err : g_create_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(ctx, call)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? ISDC_ERR_OOM : ISDC_ERR_CUDA,       \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define LAUNCH_CHECK(ctx) CUDA_TRY(ctx, cudaGetLastError())

// Events around every launch while profiling is on; the algorithmic bytes and
// FP operations of the launch (a model: each input read once, each output
// written once; one op = one add, multiply or fused multiply-add) are summed
// on the host.
void prof_flush(isdc_ctx* ctx) {
  Profiler& P = ctx->prof;
  if (!P.used) return;
  cudaEventSynchronize(P.pool[P.used - 1].e1);
  for (size_t q = 0; q < P.used; ++q) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, P.pool[q].e0, P.pool[q].e1) == cudaSuccess) P.ms[P.pool[q].cls] += t;
    else cudaGetLastError();
  }
  P.used = 0;
}

struct ProfScope {
  isdc_ctx* ctx;
  int idx = -1, gidx = -1;
  ProfScope(isdc_ctx* c, int cls, double bytes, double ops, bool fp64) : ctx(c) {
    Profiler& P = ctx->prof;
    if (!P.on) return;
    if (P.capturing) {
      P.d_launches[cls] += 1;
      P.d_bytes[cls] += bytes;
      (fp64 ? P.d_dp[cls] : P.d_sp[cls]) += ops;
      if (!(P.event_mask & (1u << cls))) return;
      if (P.gused == P.gpool.size()) {
        Profiler::Rec r{};
        if (cudaEventCreate(&r.e0) != cudaSuccess) return;
        if (cudaEventCreate(&r.e1) != cudaSuccess) { cudaEventDestroy(r.e0); return; }
        P.gpool.push_back(r);
      }
      gidx = int(P.gused++);
      P.gpool[gidx].cls = cls;
      // an external record inside a capture becomes an event-record node
      cudaEventRecordWithFlags(P.gpool[gidx].e0, ctx->stream, cudaEventRecordExternal);
      return;
    }
    P.launches[cls] += 1;
    P.bytes[cls] += bytes;
    (fp64 ? P.dp_ops[cls] : P.sp_ops[cls]) += ops;
    if (!(P.event_mask & (1u << cls))) return;
    if (P.used == P.pool.size()) {
      if (P.pool.size() >= 16384) {
        prof_flush(ctx);
      } else {
        Profiler::Rec r{};
        if (cudaEventCreate(&r.e0) != cudaSuccess) return;
        if (cudaEventCreate(&r.e1) != cudaSuccess) { cudaEventDestroy(r.e0); return; }
        P.pool.push_back(r);
      }
    }
    idx = int(P.used++);
    P.pool[idx].cls = cls;
    cudaEventRecord(P.pool[idx].e0, ctx->stream);
  }
  ~ProfScope() {
    if (idx >= 0) cudaEventRecord(ctx->prof.pool[idx].e1, ctx->stream);
    if (gidx >= 0) cudaEventRecordWithFlags(ctx->prof.gpool[gidx].e1, ctx->stream, cudaEventRecordExternal);
  }
};

// After a replay of a profiled sweep graph has completed: add its event times
// and its per-sweep counts.
void prof_graph_replayed(isdc_ctx* ctx) {
  Profiler& P = ctx->prof;
  for (size_t q = 0; q < P.gused; ++q) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, P.gpool[q].e0, P.gpool[q].e1) == cudaSuccess) P.ms[P.gpool[q].cls] += t;
    else cudaGetLastError();  // a timing failure must not surface as a later launch error
  }
  for (int c = 0; c < PC_COUNT; ++c) {
    P.launches[c] += P.d_launches[c];
    P.bytes[c] += P.d_bytes[c];
    P.dp_ops[c] += P.d_dp[c];
    P.sp_ops[c] += P.d_sp[c];
  }
}

inline double nb_ops(int dim) { return dim == 2 ? 3.0 : 5.0; }
// FP64/FP32 operations per updated point of a natural-layout red-black pass:
// 3 additions + 1 FMA in 2D; in 3D 4 additions + 1 FMA per step of a diagonal
// of zb points plus one addition for its first point (k_rbgs3).
inline double rb_ops(int dim, int zb) { return dim == 2 ? 4.0 : 5.0 + 1.0 / (zb < 0 ? -zb : zb); }

// Row scaling of H = I - a L_h on a grid of side s: c = a/h^2, d = 1 + 2 dim c,
// kappa = c / d.
struct LevelCoef {
  double c, d, kappa;
};
inline LevelCoef level_coef(int dim, int s, double a) {
  const double h = 1.0 / (s + 1), c = a / (h * h), d = 1.0 + 2.0 * dim * c;
  return {c, d, c / d};
}

inline dim3 pt_grid(int dim, int s) { return dim3((s + kBX - 1) / kBX, (s + kBY - 1) / kBY, dim == 3 ? s : 1); }
inline dim3 rb_grid(int dim, int s, int zb = 1) {
  return dim3(((s + 1) / 2 + kBX - 1) / kBX, (s + kBY - 1) / kBY, dim == 3 ? (s + zb - 1) / zb : 1);
}
const dim3 kBlock(kBX, kBY, 1);

inline size_t pow_dim(int dim, size_t s) { return dim == 2 ? s * s : s * s * s; }

// Largest side handled by the single-block bottom kernel.  One block runs on
// one SM, whose FP64 pipe issues 2 operations per clock on GB300, so FP64
// hierarchies hand only the smallest grids to it; FP32 ones go deeper.
int bottom_threshold(int dim, bool fp64) { return dim == 2 ? (fp64 ? 31 : 63) : (fp64 ? 7 : 15); }

// Entries of one dense coarsest-level inverse: side 3 (9 / 27 unknowns) on the
// Dirichlet grids, side 4 (16 / 64 unknowns) on the periodic ones.
inline size_t ainv_slot(const isdc_ctx* ctx) {
  if (ctx->equation == 1) return ctx->dim == 2 ? 256 : 4096;
  return ctx->dim == 2 ? 81 : 729;
}

template <typename T>
isdc_status alloc_hier(isdc_ctx* ctx, Hier<T>& H, bool own_level0) {
  int s = ctx->n, l = 0;
  const bool periodic = ctx->equation == 1;
  for (;;) {
    H.side[l] = s;
    H.npts[l] = pow_dim(ctx->dim, s);
    ++l;
    if (periodic ? s <= 4 : s <= 3) break;
    s = periodic ? s / 2 : (s - 1) / 2;
  }
  H.nlev = l;
  H.lb = 0;
  // levels with side <= the threshold run in one block (compact 2D: 31; periodic: 32 in 2D, 8 in 3D)
  const int thr = ctx->stencil == 1 ? 31 : periodic ? (ctx->dim == 2 ? 32 : 8) : bottom_threshold(ctx->dim, sizeof(T) == 8);
  while (H.side[H.lb] > thr) ++H.lb;
  for (int q = 0; q < H.nlev; ++q) {
    const size_t bytes = H.npts[q] * sizeof(T);
    const bool global_level = q < H.lb;
    if (q > 0 || own_level0) {
      if (global_level || q == H.lb) {
        CUDA_TRY(ctx, cudaMalloc(&H.x[q], bytes));
        CUDA_TRY(ctx, cudaMalloc(&H.b[q], bytes));
      }
    }
    if (global_level) {
      CUDA_TRY(ctx, cudaMalloc(&H.r[q], bytes));
      if (ctx->opt.smoother == ISDC_SMOOTHER_JACOBI) CUDA_TRY(ctx, cudaMalloc(&H.t[q], bytes));
    }
  }
  size_t sm = 0;
  for (int q = H.lb; q < H.nlev; ++q) sm += 3 * H.npts[q] * sizeof(T);
  H.bottom_smem = sm;
  const size_t ainv = size_t(ctx->P) * ainv_slot(ctx) * sizeof(T);
  CUDA_TRY(ctx, cudaMalloc(&H.Ainv, ainv));
  return ISDC_OK;
}

template <typename T>
void free_hier(Hier<T>& H, bool own_level0) {
  for (int q = 0; q < H.nlev; ++q) {
    if (q > 0 || own_level0) {
      cudaFree(H.x[q]);
      cudaFree(H.b[q]);
    }
    cudaFree(H.r[q]);
    cudaFree(H.t[q]);
  }
  cudaFree(H.Ainv);
}

// Upload d * H^{-1} of the side-3 grid for a = dt_m nu into a slot (it acts
// on the row-scaled right-hand side beta = b / d).
template <typename T>
isdc_status upload_ainv(isdc_ctx* ctx, Hier<T>& H, int slot, double a) {
  std::vector<double> inv;
  double d3;
  if (ctx->stencil == 1) {  // c0 (W - a L_9)^{-1}, c0 = 2/3 + 10 a / (3 h^2), h = 1/4
    coarse_inverse9(a, inv);
    d3 = 2.0 / 3.0 + 10.0 * a * 16.0 / 3.0;
  } else if (ctx->equation == 1) {  // periodic side 4, h = 1/2
    coarse_inverse_per(ctx->dim, a, inv);
    d3 = 1.0 + 2.0 * ctx->dim * a * 4.0;
  } else {
    coarse_inverse(ctx->dim, a, inv);
    d3 = 1.0 + 2.0 * ctx->dim * a * 16.0;  // h = 1/4 on the side-3 grid
  }
  std::vector<T> tv(inv.size());
  for (size_t q = 0; q < inv.size(); ++q) tv[q] = T(d3 * inv[q]);
  const size_t each = ainv_slot(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(H.Ainv + slot * each, tv.data(), each * sizeof(T), cudaMemcpyHostToDevice,
                                ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // tv is a host temporary
  return ISDC_OK;
}

template <typename T, int DIM>
void configure_bottom(const Hier<T>& H) {
  cudaFuncSetAttribute(k_bottom<T, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(H.bottom_smem));
}

// ---------------------------------------------------------------------------
// V-cycle on (I - a L_h) x = b (textbook geometric multigrid; the paper's
// solver is not described).  x0/b0 are the level-0 arrays in precision T.
// ---------------------------------------------------------------------------
template <typename T, int DIM>
isdc_status smooth_level(isdc_ctx* ctx, Hier<T>& H, int l, double a, T*& x, T* home, const T* b, bool& zero,
                         int sweeps) {
  // x: where the level's iterate lives now; home: its own array (Jacobi
  // ping-pongs between home and H.t[l]).
  const int s = H.side[l];
  const T kappa = T(level_coef(DIM, s, a).kappa);
  const int zb = ctx->zbl[l];
  for (int it = 0; it < sweeps; ++it) {
    if (ctx->opt.smoother == ISDC_SMOOTHER_JACOBI) {
      T* out = (x == H.t[l]) ? home : H.t[l];
      {
        const double Np = double(H.npts[l]);
        ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, (zero ? 2.0 : 3.0) * Np * sizeof(T),
                     (zero ? 1.0 : nb_ops(DIM) + 3.0) * Np, sizeof(T) == 8);
        k_jacobi<T, DIM><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, kappa, T(ctx->opt.omega), x, b, out,
                                                                        zero ? 1 : 0);
      }
      LAUNCH_CHECK(ctx);
      x = out;
    } else {
      const double Np = double(H.npts[l]);
      {
        ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, (zero ? 1.0 : 1.5) * Np * sizeof(T),
                     (zero ? 0.0 : rb_ops(DIM, zb)) * 0.5 * Np, sizeof(T) == 8);
        launch_rbgs<T, DIM>(ctx->stream, s, kappa, 0, x, b, zero, zb);
      }
      LAUNCH_CHECK(ctx);
      {
        ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, 1.5 * Np * sizeof(T), rb_ops(DIM, zb) * 0.5 * Np,
                     sizeof(T) == 8);
        launch_rbgs<T, DIM>(ctx->stream, s, kappa, 1, x, b, false, zb);
      }
      LAUNCH_CHECK(ctx);
    }
    zero = false;
  }
  return ISDC_OK;
}

// V-cycle from level l0 (default the fine level) down and back; x0/b0 are
// level l0's unknown and scaled right-hand side.
template <typename T, int DIM>
isdc_status vcycle(isdc_ctx* ctx, Hier<T>& H, int slot, double a, T* x0, const T* b0, bool zero0, int l0 = 0) {
  T* xcur[kMaxLevels];
  isdc_status st;
  // downward leg on the levels above the bottom block
  for (int l = l0; l < H.lb; ++l) {
    T* home = (l == l0) ? x0 : H.x[l];
    T* x = home;
    const T* b = (l == l0) ? b0 : H.b[l];
    bool zero = (l == l0) ? zero0 : true;
    const int s = H.side[l];
    if (ctx->opt.nu1 == 0 && zero) {
      CUDA_TRY(ctx, cudaMemsetAsync(x, 0, H.npts[l] * sizeof(T), ctx->stream));
      zero = false;
    }
    if ((st = smooth_level<T, DIM>(ctx, H, l, a, x, home, b, zero, ctx->opt.nu1)) != ISDC_OK) return st;
    const LevelCoef lf = level_coef(DIM, s, a);
    const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
    // after a complete red-black sweep only the red rows carry a residual
    const bool red_only = ctx->opt.smoother == ISDC_SMOOTHER_RBGS && ctx->opt.nu1 >= 1;
    const int kc = (sizeof(T) == 8 ? ctx->rr64 : ctx->rr32)[l];
    if (kc > 0) {
      // residual and full weighting in one launch: r stays in shared memory
      const int sc = H.side[l + 1];
      const T ws = T(lf.d / (level_coef(DIM, sc, a).d * (DIM == 2 ? 16.0 : 64.0)));
      const double f = red_only ? 0.5 : 1.0;
      ProfScope ps(ctx, l == 0 ? PC_RESRESTRICT0 : PC_RESRESTRICTC, ((red_only ? 1.5 : 2.0) * Np + Nc) * sizeof(T),
                   (nb_ops(DIM) + 2.0) * f * Np +
                       (red_only ? (DIM == 2 ? 6.0 : 15.0) : (DIM == 2 ? 9.0 : 27.0)) * Nc,
                   sizeof(T) == 8);
      const dim3 g = resrestrict_grid(DIM, sc, kc), blk(kRrTX, kRrTY, 1);
      if (red_only)
        k_resrestrict<T, DIM, true><<<g, blk, 0, ctx->stream>>>(sc, T(lf.kappa), ws, x, b, H.b[l + 1], kc);
      else
        k_resrestrict<T, DIM, false><<<g, blk, 0, ctx->stream>>>(sc, T(lf.kappa), ws, x, b, H.b[l + 1], kc);
      LAUNCH_CHECK(ctx);
      xcur[l] = x;
      continue;
    }
    {
      const double f = red_only ? 0.5 : 1.0;
      ProfScope ps(ctx, l == 0 ? PC_RESIDUAL0 : PC_RESIDUALC, (red_only ? 2.0 : 3.0) * Np * sizeof(T),
                   (nb_ops(DIM) + 2.0) * f * Np, sizeof(T) == 8);
      if (red_only)
        k_residual<T, DIM, true><<<rb_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, T(lf.kappa), x, b, H.r[l]);
      else
        k_residual<T, DIM, false><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, T(lf.kappa), x, b, H.r[l]);
    }
    LAUNCH_CHECK(ctx);
    const int sc = H.side[l + 1];
    {
      const T ws = T(lf.d / (level_coef(DIM, sc, a).d * (DIM == 2 ? 16.0 : 64.0)));
      ProfScope ps(ctx, l == 0 ? PC_RESTRICT0 : PC_RESTRICTC, ((red_only ? 0.5 : 1.0) * Np + Nc) * sizeof(T),
                   (red_only ? (DIM == 2 ? 6.0 : 15.0) : (DIM == 2 ? 9.0 : 27.0)) * Nc, sizeof(T) == 8);
      if (red_only)
        k_restrict<T, DIM, true><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
      else
        k_restrict<T, DIM, false><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
    }
    LAUNCH_CHECK(ctx);
    xcur[l] = x;
  }
  // bottom levels in one block
  {
    BottomParams<T> P{};
    P.nlev = H.nlev - H.lb;
    for (int q = 0; q < P.nlev; ++q) {
      const int s = H.side[H.lb + q];
      const LevelCoef lf = level_coef(DIM, s, a);
      P.side[q] = s;
      P.kappa[q] = T(lf.kappa);
      P.rscale[q] = q + 1 < P.nlev
                        ? T(lf.d / (level_coef(DIM, H.side[H.lb + q + 1], a).d * (DIM == 2 ? 16.0 : 64.0)))
                        : T(0);
    }
    P.smoother = ctx->opt.smoother;
    P.nu1 = ctx->opt.nu1;
    P.nu2 = ctx->opt.nu2;
    P.omega = T(ctx->opt.omega);
    P.Ainv = H.Ainv + size_t(slot) * (DIM == 2 ? 81 : 729);
    const T* bb = H.lb == l0 ? b0 : H.b[H.lb];
    T* xb = H.lb == l0 ? x0 : H.x[H.lb];
    const int load_x = (H.lb == l0 && !zero0) ? 1 : 0;
    {
      ProfScope ps(ctx, PC_BOTTOM, (2.0 + load_x) * double(H.npts[H.lb]) * sizeof(T), 0.0, sizeof(T) == 8);
      k_bottom<T, DIM><<<1, kBottomThreads, H.bottom_smem, ctx->stream>>>(P, bb, xb, load_x);
    }
    LAUNCH_CHECK(ctx);
    xcur[H.lb] = xb;
  }
  // upward leg
  for (int l = H.lb - 1; l >= l0; --l) {
    const int sc = H.side[l + 1], s = H.side[l];
    T* home = (l == l0) ? x0 : H.x[l];
    T* x = xcur[l];
    {
      // a red half sweep follows: it overwrites the red points, so correct the black ones only
      const bool black_only = ctx->opt.smoother == ISDC_SMOOTHER_RBGS && ctx->opt.nu2 >= 1;
      const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
      ProfScope ps(ctx, l == 0 ? PC_PROLONG0 : PC_PROLONGC, ((black_only ? 1.0 : 2.0) * Np + Nc) * sizeof(T),
                   (black_only ? (DIM == 2 ? 1.25 : 1.75) : (DIM == 2 ? 2.0 : 2.5)) * Np, sizeof(T) == 8);
      if (black_only)
        k_prolong_add<T, DIM, true><<<pt_grid(DIM, sc + 1), kBlock, 0, ctx->stream>>>(sc, xcur[l + 1], x);
      else
        k_prolong_add<T, DIM, false><<<pt_grid(DIM, sc + 1), kBlock, 0, ctx->stream>>>(sc, xcur[l + 1], x);
    }
    LAUNCH_CHECK(ctx);
    bool zero = false;
    if ((st = smooth_level<T, DIM>(ctx, H, l, a, x, home, l == l0 ? b0 : H.b[l], zero, ctx->opt.nu2)) != ISDC_OK)
      return st;
    xcur[l] = x;
  }
  if (xcur[l0] != x0)
    CUDA_TRY(ctx, cudaMemcpyAsync(x0, xcur[l0], H.npts[l0] * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
  return ISDC_OK;
}

// One colour pass on the split fine level with zb z-planes per thread.
// Rows of the split layout hold H = (n+1)/2 slots, a power of two; from
// H = 4 on the 4-slot form applies.
template <int DIM>
void launch_rbgs_split(cudaStream_t st, int zb, int s, float kappa, int colour, float* xc, const float* xo,
                       const float* bc, bool zero) {
  const int z = zero ? 1 : 0, H = (s + 1) / 2;
  const int zbe = DIM == 3 ? zb : 1;
  if (H % 4 != 0) {
    const dim3 g = rb_grid(DIM, s, 1);
    k_rbgs_split<DIM, 1><<<g, kBlock, 0, st>>>(s, kappa, colour, xc, xo, bc, z);
    return;
  }
  const dim3 g(unsigned((H / 4 + kBX - 1) / kBX), unsigned((s + kBY - 1) / kBY),
               unsigned(DIM == 3 ? (s + zbe - 1) / zbe : 1));
  if (DIM == 2 || zb <= 1) k_rbgs_split4<DIM, 1><<<g, kBlock, 0, st>>>(s, kappa, colour, xc, xo, bc, z);
  else if (zb == 2) k_rbgs_split4<DIM, 2><<<g, kBlock, 0, st>>>(s, kappa, colour, xc, xo, bc, z);
  else if (zb == 4) k_rbgs_split4<DIM, 4><<<g, kBlock, 0, st>>>(s, kappa, colour, xc, xo, bc, z);
  else k_rbgs_split4<DIM, 8><<<g, kBlock, 0, st>>>(s, kappa, colour, xc, xo, bc, z);
}

// One blocked pass of `depth` red-black sweeps on the split fine level (3D):
// black read from xb_in, red written in place, black written to xb_out.
inline void launch_rbgs_tb(cudaStream_t st, int depth, int zc, int s, float kappa, const float* xb_in, float* xr,
                           float* xb_out, const float* br, const float* bb, bool zero) {
  const dim3 g(unsigned(((s + 1) / 2 + kTbX - 1) / kTbX), unsigned((s + kTbY - 1) / kTbY), unsigned((s + zc - 1) / zc));
  if (depth == 1)
    k_rbgs_split_tb<2><<<g, kTbThreads, TbShape<2>::smem_bytes, st>>>(s, kappa, xb_in, xr, xb_out, br, bb,
                                                                       zero ? 1 : 0, zc);
  else
    k_rbgs_split_tb<4><<<g, kTbThreads, TbShape<4>::smem_bytes, st>>>(s, kappa, xb_in, xr, xb_out, br, bb,
                                                                       zero ? 1 : 0, zc);
}

// nsw red-black sweeps on the split fine level (the first from a zero guess
// if `zero`).  *xb is the array holding the black values; blocked passes
// move them to the other black array.
template <int DIM>
isdc_status smooth_split(isdc_ctx* ctx, float kappa, int nsw, bool zero, float** xb) {
  const int s = ctx->n;
  const size_t hn = ctx->hn;
  float *x0 = ctx->sp_x, *b0 = ctx->sp_b, *b1 = ctx->sp_b + hn;
  const double Np = double(ctx->N);
  const double pass_ops = (nb_ops(DIM) + 1.0) * 0.5 * Np;
  if (DIM == 3 && ctx->tb_depth > 0) {
    while (nsw > 0) {
      const int d = std::min(nsw, ctx->tb_depth);
      float* xo = *xb == ctx->sp_xb ? ctx->sp_x + hn : ctx->sp_xb;
      {
        ProfScope ps(ctx, PC_SMOOTH0, (zero ? 2.0 : 2.5) * Np * 4, (2.0 * d - (zero ? 1.0 : 0.0)) * pass_ops, false);
        launch_rbgs_tb(ctx->stream, d, ctx->tb_zc, s, kappa, *xb, x0, xo, b0, b1, zero);
      }
      LAUNCH_CHECK(ctx);
      *xb = xo;
      zero = false;
      nsw -= d;
    }
    return ISDC_OK;
  }
  for (int it = 0; it < nsw; ++it, zero = false) {
    {
      ProfScope ps(ctx, PC_SMOOTH0, (zero ? 1.0 : 1.5) * Np * 4, zero ? 0.0 : pass_ops, false);
      launch_rbgs_split<DIM>(ctx->stream, ctx->zb32, s, kappa, 0, x0, *xb, b0, zero);
    }
    LAUNCH_CHECK(ctx);
    {
      ProfScope ps(ctx, PC_SMOOTH0, 1.5 * Np * 4, pass_ops, false);
      launch_rbgs_split<DIM>(ctx->stream, ctx->zb32, s, kappa, 1, *xb, x0, b1, false);
    }
    LAUNCH_CHECK(ctx);
  }
  return ISDC_OK;
}

// FP32 V-cycles with red-black smoothing whose fine level is in the
// colour-split layout (levels below it are natural): defect, n_cycles
// V-cycles on the error equation, update.  Needs nu1, nu2 >= 1.
template <int DIM>
isdc_status node_solve_split(isdc_ctx* ctx, int slot, double a, double* x, const double* beta, int n_cycles,
                             bool defect_ready) {
  const int s = ctx->n, sc = ctx->h32.side[1];
  Hier<float>& H = ctx->h32;
  const size_t hn = ctx->hn;
  float *x0 = ctx->sp_x, *xb = ctx->sp_x + hn, *b0 = ctx->sp_b, *b1 = ctx->sp_b + hn;
  const LevelCoef lf = level_coef(DIM, s, a);
  const float kappa = float(lf.kappa);
  const float ws = float(lf.d / (level_coef(DIM, sc, a).d * (DIM == 2 ? 16.0 : 64.0)));
  const double Np = double(ctx->N), Nc = double(H.npts[1]);
  const dim3 g = rb_grid(DIM, s);
  isdc_status st;
  if (!defect_ready) {
    {
      ProfScope ps(ctx, PC_DEFECT, 20.0 * Np, (nb_ops(DIM) + 2.0) * Np, true);
      k_defect_split<DIM><<<g, kBlock, 0, ctx->stream>>>(s, lf.kappa, x, beta, b0, b1);
    }
    LAUNCH_CHECK(ctx);
  }
  for (int c = 0; c < n_cycles; ++c) {
    if ((st = smooth_split<DIM>(ctx, kappa, ctx->opt.nu1, c == 0, &xb)) != ISDC_OK) return st;
    if (ctx->rr_split > 0) {
      const int kc = ctx->rr_split;
      ProfScope ps(ctx, PC_RESRESTRICT0, (1.5 * Np + Nc) * 4,
                   (nb_ops(DIM) + 2.0) * 0.5 * Np + (DIM == 2 ? 6.0 : 15.0) * Nc, false);
      k_resrestrict_red_split<DIM><<<resrestrict_grid(DIM, sc, kc), dim3(kRrTX, kRrTY, 1), 0, ctx->stream>>>(
          sc, kappa, ws, x0, xb, b0, H.b[1], kc);
    } else {
      {
        ProfScope ps(ctx, PC_RESIDUAL0, 2.0 * Np * 4, (nb_ops(DIM) + 2.0) * 0.5 * Np, false);
        k_residual_red_split<DIM><<<g, kBlock, 0, ctx->stream>>>(s, kappa, x0, xb, b0, ctx->sp_r);
      }
      LAUNCH_CHECK(ctx);
      ProfScope ps(ctx, PC_RESTRICT0, (0.5 * Np + Nc) * 4, (DIM == 2 ? 6.0 : 15.0) * Nc, false);
      k_restrict_red_split<DIM><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, ctx->sp_r, H.b[1]);
    }
    LAUNCH_CHECK(ctx);
    if ((st = vcycle<float, DIM>(ctx, H, slot, a, H.x[1], H.b[1], true, 1)) != ISDC_OK) return st;
    {
      ProfScope ps(ctx, PC_PROLONG0, (Np + Nc) * 4, (DIM == 2 ? 1.25 : 1.75) * Np, false);
      k_prolong_black_split<DIM><<<pt_grid(DIM, sc + 1), kBlock, 0, ctx->stream>>>(sc, H.x[1], x0, xb);
    }
    LAUNCH_CHECK(ctx);
    if ((st = smooth_split<DIM>(ctx, kappa, ctx->opt.nu2, false, &xb)) != ISDC_OK) return st;
  }
  {
    ProfScope ps(ctx, PC_UPDATE, 20.0 * Np, 1.0 * Np, true);
    k_update_split<DIM><<<g, kBlock, 0, ctx->stream>>>(s, x, x0, xb);
  }
  LAUNCH_CHECK(ctx);
  return ISDC_OK;
}

// n_cycles V-cycles of one node solve on (I - a L_h) x = b, x an FP64 device
// array, beta = b/d.  FP64 mode: V-cycles on x.  FP32 mode (defect
// correction): the fine-level residual of the node equation in FP64, rounded
// to FP32, n_cycles FP32 V-cycles on the error equation from e = 0, and one
// FP64 update x += e.  defect_ready: the scaled FP32 defect is already in the
// fine level's rhs (k_rhs_defect), beta is not read.
template <int DIM>
isdc_status node_solve(isdc_ctx* ctx, int slot, double a, double* x, const double* beta, int n_cycles,
                       bool defect_ready = false) {
  isdc_status st;
  if (!ctx->opt.vcycle_fp32) {
    for (int c = 0; c < n_cycles; ++c)
      if ((st = vcycle<double, DIM>(ctx, ctx->h64, slot, a, x, beta, false)) != ISDC_OK) return st;
    return ISDC_OK;
  }
  if (n_cycles <= 0) return ISDC_OK;
  if (ctx->sp_x) return node_solve_split<DIM>(ctx, slot, a, x, beta, n_cycles, defect_ready);
  const int s = ctx->n;
  Hier<float>& H = ctx->h32;
  const double Np = double(ctx->N);
  if (!defect_ready) {
    {
      ProfScope ps(ctx, PC_DEFECT, 20.0 * Np, (nb_ops(DIM) + 2.0) * Np, true);
      k_defect<DIM><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, level_coef(DIM, s, a).kappa, x, beta, H.b[0]);
    }
    LAUNCH_CHECK(ctx);
  }
  for (int c = 0; c < n_cycles; ++c)
    if ((st = vcycle<float, DIM>(ctx, H, slot, a, H.x[0], H.b[0], c == 0)) != ISDC_OK) return st;
  {
    ProfScope ps(ctx, PC_UPDATE, 20.0 * Np, 1.0 * Np, true);
    k_update<DIM><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, x, H.x[0]);
  }
  LAUNCH_CHECK(ctx);
  return ISDC_OK;
}

// ---------------------------------------------------------------------------
// 4th-order compact stencil (Sec. 3, Eq. 5), 2D, FP64: multigrid on
// (W - a L_9) x = b and the sweep pieces that differ from W = I.
// ---------------------------------------------------------------------------
struct Coef9 {
  double c0, ke, kc;  // diagonal; row-scaled edge and corner couplings
};
inline Coef9 coef9(int s, double a) {
  const double h = 1.0 / (s + 1), q = a / (6.0 * h * h);
  const double c0 = 2.0 / 3.0 + 20.0 * q, ce = 1.0 / 12.0 - 4.0 * q, cc = -q;
  return {c0, -ce / c0, -cc / c0};
}

// Damped-Jacobi sweeps on level l (x ping-pongs between home and H.t[l]).
isdc_status smooth_level9(isdc_ctx* ctx, Hier<double>& H, int l, double a, double*& x, double* home, const double* b,
                          bool& zero, int sweeps) {
  const int s = H.side[l];
  const Coef9 k = coef9(s, a);
  for (int it = 0; it < sweeps; ++it) {
    double* out = (x == H.t[l]) ? home : H.t[l];
    {
      const double Np = double(H.npts[l]);
      ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, (zero ? 2.0 : 3.0) * Np * 8, (zero ? 1.0 : 12.0) * Np, true);
      k_jacobi9<double><<<pt_grid(2, s), kBlock, 0, ctx->stream>>>(s, k.ke, k.kc, ctx->opt.omega, x, b, out,
                                                                   zero ? 1 : 0);
    }
    LAUNCH_CHECK(ctx);
    x = out;
    zero = false;
  }
  return ISDC_OK;
}

// One V-cycle on the row-scaled compact system x - ke E - kc C = beta.
isdc_status vcycle9(isdc_ctx* ctx, int slot, double a, double* x0, const double* b0) {
  Hier<double>& H = ctx->h64;
  double* xcur[kMaxLevels];
  isdc_status st;
  for (int l = 0; l < H.lb; ++l) {
    double* home = l == 0 ? x0 : H.x[l];
    double* x = home;
    const double* b = l == 0 ? b0 : H.b[l];
    bool zero = l > 0;
    const int s = H.side[l], sc = H.side[l + 1];
    if (ctx->opt.nu1 == 0 && zero) {
      CUDA_TRY(ctx, cudaMemsetAsync(x, 0, H.npts[l] * sizeof(double), ctx->stream));
      zero = false;
    }
    if ((st = smooth_level9(ctx, H, l, a, x, home, b, zero, ctx->opt.nu1)) != ISDC_OK) return st;
    const Coef9 k = coef9(s, a);
    const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
    {
      ProfScope ps(ctx, l == 0 ? PC_RESIDUAL0 : PC_RESIDUALC, 3.0 * Np * 8, 11.0 * Np, true);
      k_residual9<double><<<pt_grid(2, s), kBlock, 0, ctx->stream>>>(s, k.ke, k.kc, x, b, H.r[l]);
    }
    LAUNCH_CHECK(ctx);
    {
      const double ws = k.c0 / (coef9(sc, a).c0 * 16.0);
      ProfScope ps(ctx, l == 0 ? PC_RESTRICT0 : PC_RESTRICTC, (Np + Nc) * 8, 9.0 * Nc, true);
      k_restrict<double, 2, false><<<pt_grid(2, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
    }
    LAUNCH_CHECK(ctx);
    xcur[l] = x;
  }
  {  // the levels with side <= 31 in one block, the side-3 one by the dense inverse
    BottomParams9 B{};
    B.nlev = H.nlev - H.lb;
    for (int q = 0; q < B.nlev; ++q) {
      const int s = H.side[H.lb + q];
      const Coef9 k = coef9(s, a);
      B.side[q] = s;
      B.ke[q] = k.ke;
      B.kc[q] = k.kc;
      B.rscale[q] = q + 1 < B.nlev ? k.c0 / (coef9(H.side[H.lb + q + 1], a).c0 * 16.0) : 0.0;
    }
    B.nu1 = ctx->opt.nu1;
    B.nu2 = ctx->opt.nu2;
    B.omega = ctx->opt.omega;
    B.G = H.Ainv + size_t(slot) * 81;
    const double* bb = H.lb == 0 ? b0 : H.b[H.lb];
    double* xb = H.lb == 0 ? x0 : H.x[H.lb];
    ProfScope ps(ctx, PC_BOTTOM, 2.0 * double(H.npts[H.lb]) * 8, 0.0, true);
    k_bottom9<<<1, kBottomThreads, H.bottom_smem, ctx->stream>>>(B, bb, xb, H.lb == 0 ? 1 : 0);
    LAUNCH_CHECK(ctx);
    xcur[H.lb] = xb;
  }
  for (int l = H.lb - 1; l >= 0; --l) {
    const int sc = H.side[l + 1];
    double* home = l == 0 ? x0 : H.x[l];
    double* x = xcur[l];
    {
      const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
      ProfScope ps(ctx, l == 0 ? PC_PROLONG0 : PC_PROLONGC, (2.0 * Np + Nc) * 8, 2.0 * Np, true);
      k_prolong_add<double, 2, false><<<pt_grid(2, sc + 1), kBlock, 0, ctx->stream>>>(sc, xcur[l + 1], x);
    }
    LAUNCH_CHECK(ctx);
    bool zero = false;
    if ((st = smooth_level9(ctx, H, l, a, x, home, l == 0 ? b0 : H.b[l], zero, ctx->opt.nu2)) != ISDC_OK) return st;
    xcur[l] = x;
  }
  if (xcur[0] != x0)
    CUDA_TRY(ctx, cudaMemcpyAsync(x0, xcur[0], H.npts[0] * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return ISDC_OK;
}

isdc_status node_residual_norm9(isdc_ctx* ctx, double a, const double* x, const double* b, double* out) {
  const int s = ctx->n;
  const Coef9 k = coef9(s, a);
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal + 1, 0, sizeof(unsigned long long), ctx->stream));
  {
    ProfScope ps(ctx, PC_RESNORM, 16.0 * double(ctx->N), 13.0 * double(ctx->N), true);
    k_resnorm9<<<pt_grid(2, s), kBlock, 0, ctx->stream>>>(s, k.ke, k.kc, k.c0, x, b, ctx->d_scal + 1);
  }
  LAUNCH_CHECK(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned long long bits = ctx->h_scal[1];
  std::memcpy(out, &bits, sizeof(double));
  return ISDC_OK;
}

// W^{-1} of `count` arrays rho (each N) by the Chebyshev semi-iteration on the
// Jacobi splitting r <- (3/2) rho - E(r)/8 (W = (2/3)(I + E/8); the Jacobi
// iteration matrix -E/8 has its spectrum inside [-1/2, 1/2]), starting from 0:
// after k steps the error is at most 2 / T_k(2) of the initial one in the
// 2-norm (T_k the Chebyshev polynomial), against 2^-k for plain Jacobi steps
// at three quarters of the traffic per step.  The result is in *res (one of the
// two scratch sets; each step overwrites the iterate two steps back).
constexpr int kWinvSweepIters = 12;  // residual for the stopping test: 2 / T_12(2) = 5.4e-7 relative
constexpr int kWinvEndIters = 29;    // Gauss-Legendre end value: 2 / T_29(2) below FP64 rounding
isdc_status w_inverse(isdc_ctx* ctx, int count, const double* rho, double* s0, double* s1, int iters,
                      const double** res) {
  const int n = ctx->n;
  const size_t N = ctx->N;
  const dim3 g(unsigned((n + kBX - 1) / kBX), unsigned((n + kBY - 1) / kBY), unsigned(count));
  {
    ProfScope ps(ctx, PC_WINV, 2.0 * 8.0 * double(N) * count, 1.0 * double(N) * count, true);
    k_winv_jacobi<<<g, kBlock, 0, ctx->stream>>>(n, N, rho, nullptr, s0);  // y_1 = (3/2) rho
  }
  LAUNCH_CHECK(ctx);
  const double* prev = nullptr;  // y_{k-1} (y_0 = 0)
  double* cur = s0;              // y_k
  double omega = 1.0;
  for (int k = 1; k < iters; ++k) {
    omega = k == 1 ? 2.0 / (2.0 - 0.25) : 1.0 / (1.0 - 0.0625 * omega);  // rho^2 = 1/4
    double* out = prev ? const_cast<double*>(prev) : s1;
    {
      ProfScope ps(ctx, PC_WINV, (prev ? 4.0 : 3.0) * 8.0 * double(N) * count, 8.0 * double(N) * count, true);
      k_winv_cheb<<<g, kBlock, 0, ctx->stream>>>(n, N, omega, rho, cur, prev, out);
    }
    LAUNCH_CHECK(ctx);
    prev = cur;
    cur = out;
  }
  *res = cur;
  return ISDC_OK;
}

template <int OFF, int P>
void launch_sweep_end9_p(isdc_ctx* ctx, double nu6) {
  k_sweep_end9<OFF, P><<<pt_grid(2, ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, ctx->N, nu6, ctx->opt.reaction,
                                                                       ctx->tables, ctx->U, ctx->F, ctx->G, ctx->C,
                                                                       ctx->Rs);
}

// End of a compact sweep: f~ at the last point, the W-weighted residuals, the
// next C_m; then W^{-1} of the residuals and their max norm into d_scal[0].
isdc_status sweep_end9(isdc_ctx* ctx) {
  const int P = ctx->P;
  const size_t N = ctx->N;
  const double nu6 = ctx->nu / (6.0 * ctx->h * ctx->h);
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal, 0, sizeof(unsigned long long), ctx->stream));
  {
    const double Pd = P, M = ctx->M, Np = double(N);
    ProfScope ps(ctx, PC_SWEEP_END, (2.0 * Pd + 2.0 * (Pd - 1.0) + (Pd - 1.0) + 2.0) * 8.0 * Np,
                 (30.0 + (Pd - 1.0) * (M + 8.0) + 4.0 * (Pd - 1.0)) * Np, true);
    if (ctx->off) {
      switch (P) {
        case 3: launch_sweep_end9_p<1, 3>(ctx, nu6); break;
        case 4: launch_sweep_end9_p<1, 4>(ctx, nu6); break;
        case 5: launch_sweep_end9_p<1, 5>(ctx, nu6); break;
        case 6: launch_sweep_end9_p<1, 6>(ctx, nu6); break;
        case 7: launch_sweep_end9_p<1, 7>(ctx, nu6); break;
        default: launch_sweep_end9_p<1, 8>(ctx, nu6); break;
      }
    } else {
      switch (P) {
        case 2: launch_sweep_end9_p<0, 2>(ctx, nu6); break;
        case 3: launch_sweep_end9_p<0, 3>(ctx, nu6); break;
        case 4: launch_sweep_end9_p<0, 4>(ctx, nu6); break;
        case 5: launch_sweep_end9_p<0, 5>(ctx, nu6); break;
        case 6: launch_sweep_end9_p<0, 6>(ctx, nu6); break;
        default: launch_sweep_end9_p<0, 7>(ctx, nu6); break;
      }
    }
  }
  LAUNCH_CHECK(ctx);
  const size_t R = size_t(P - 1) * N;
  const double* r = nullptr;
  isdc_status st = w_inverse(ctx, P - 1, ctx->Rs, ctx->Rs + R, ctx->Rs + 2 * R, kWinvSweepIters, &r);
  if (st != ISDC_OK) return st;
  {
    ProfScope ps(ctx, PC_WINV, double(R) * 8, 0.0, true);
    k_maxabs<<<4 * 152, 256, 0, ctx->stream>>>(R, r, ctx->d_scal);
  }
  LAUNCH_CHECK(ctx);
  return ISDC_OK;
}

template <int DIM>
isdc_status node_residual_norm(isdc_ctx* ctx, double a, const double* x, const double* b, double* out) {
  const int s = ctx->n;
  const LevelCoef lf = level_coef(DIM, s, a);
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal + 1, 0, sizeof(unsigned long long), ctx->stream));
  {
    ProfScope ps(ctx, PC_RESNORM, 16.0 * double(ctx->N), (nb_ops(DIM) + 3.0) * double(ctx->N), true);
    k_resnorm<DIM><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, lf.kappa, lf.d, x, b, ctx->d_scal + 1);
  }
  LAUNCH_CHECK(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned long long bits = ctx->h_scal[1];
  std::memcpy(out, &bits, sizeof(double));
  return ISDC_OK;
}

inline double bits_to_double(unsigned long long b) {
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
}

// k_sweep_end for the context's point count (compile-time P: straight-line
// code, registers for exactly P points).
template <int DIM, int OFF, int P>
void launch_sweep_end_p(isdc_ctx* ctx, double nu_h2) {
  k_sweep_end<DIM, OFF, P><<<pt_grid(DIM, ctx->n), kBlock, 0, ctx->stream>>>(
      ctx->n, ctx->N, nu_h2, ctx->opt.reaction, ctx->cprime, ctx->tables, ctx->U, ctx->F, ctx->FE, ctx->C,
      ctx->d_scal);
}

template <int DIM>
void launch_sweep_end(isdc_ctx* ctx, double nu_h2) {
  if (ctx->off) {
    switch (ctx->P) {
      case 3: launch_sweep_end_p<DIM, 1, 3>(ctx, nu_h2); break;
      case 4: launch_sweep_end_p<DIM, 1, 4>(ctx, nu_h2); break;
      case 5: launch_sweep_end_p<DIM, 1, 5>(ctx, nu_h2); break;
      case 6: launch_sweep_end_p<DIM, 1, 6>(ctx, nu_h2); break;
      case 7: launch_sweep_end_p<DIM, 1, 7>(ctx, nu_h2); break;
      default: launch_sweep_end_p<DIM, 1, 8>(ctx, nu_h2); break;
    }
  } else {
    switch (ctx->P) {
      case 2: launch_sweep_end_p<DIM, 0, 2>(ctx, nu_h2); break;
      case 3: launch_sweep_end_p<DIM, 0, 3>(ctx, nu_h2); break;
      case 4: launch_sweep_end_p<DIM, 0, 4>(ctx, nu_h2); break;
      case 5: launch_sweep_end_p<DIM, 0, 5>(ctx, nu_h2); break;
      case 6: launch_sweep_end_p<DIM, 0, 6>(ctx, nu_h2); break;
      default: launch_sweep_end_p<DIM, 0, 7>(ctx, nu_h2); break;
    }
  }
}

template <int DIM>
isdc_status sweep_end(isdc_ctx* ctx) {
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal, 0, sizeof(unsigned long long), ctx->stream));
  const double nu_h2 = ctx->nu / (ctx->h * ctx->h);
  {
    const double M = ctx->M, P = ctx->P, Np = double(ctx->N);
    // reads P u, M-1 f, P-1 f^E; writes f_{P-1} and P-1 C.  Ops: f_{P-1}: nb+2;
    // f^E of the last point: 2; dt Q f: (P-1)M; residual: 2(P-1); C: 4(P-1) - 1
    // (C': 3(P-1) - 1)
    ProfScope ps(ctx, PC_SWEEP_END, (3.0 * P + M - 2.0) * 8.0 * Np,
                 (nb_ops(DIM) + 4.0 + (P - 1.0) * M + (ctx->cprime ? 5.0 : 6.0) * (P - 1.0) - 1.0) * Np, true);
    launch_sweep_end<DIM>(ctx, nu_h2);
  }
  LAUNCH_CHECK(ctx);
  return ISDC_OK;
}

// ---------------------------------------------------------------------------
// Viscous Burgers on the periodic grid (Sec. 4.1), FP64: multigrid on
// (I - a L_h) x = b with periodic kernels, and the sweep with stored f^E.
// ---------------------------------------------------------------------------
// Algorithmic FP64 operations of the WENO5 advection per point and axis: one
// face flux (the split fluxes at 6 points: 25; two reconstructions of 42
// add/multiply/FMA/divide each, one division among them; their sum) and the
// scaled difference of the point's two faces (2).
constexpr double kWenoOps = 112.0;

inline LevelCoef coef_per(int dim, int s, double a) {
  const double h = 2.0 / s, c = a / (h * h), d = 1.0 + 2.0 * dim * c;
  return {c, d, c / d};
}
inline dim3 pp_grid(int dim, int s) { return dim3((s + kBX - 1) / kBX, (s + kBY - 1) / kBY, dim == 3 ? s : 1); }
inline dim3 prb_grid(int dim, int s) {
  return dim3((s / 2 + kBX - 1) / kBX, (s + kBY - 1) / kBY, dim == 3 ? s : 1);
}

template <int DIM>
isdc_status smooth_level_per(isdc_ctx* ctx, Hier<double>& H, int l, double a, double*& x, double* home,
                             const double* b, bool& zero, int sweeps) {
  const int s = H.side[l];
  const double kappa = coef_per(DIM, s, a).kappa;
  const double Np = double(H.npts[l]);
  for (int it = 0; it < sweeps; ++it) {
    if (ctx->opt.smoother == ISDC_SMOOTHER_JACOBI) {
      double* out = (x == H.t[l]) ? home : H.t[l];
      {
        ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, (zero ? 2.0 : 3.0) * Np * 8,
                     (zero ? 1.0 : nb_ops(DIM) + 3.0) * Np, true);
        k_jacobi_per<double, DIM><<<pp_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, kappa, ctx->opt.omega, x, b, out,
                                                                                zero ? 1 : 0);
      }
      LAUNCH_CHECK(ctx);
      x = out;
    } else {
      for (int colour = 0; colour < 2; ++colour) {
        {
          const bool z = zero && colour == 0;
          ProfScope ps(ctx, l == 0 ? PC_SMOOTH0 : PC_SMOOTHC, (z ? 1.0 : 1.5) * Np * 8,
                       (z ? 0.0 : nb_ops(DIM) + 1.0) * 0.5 * Np, true);
          k_rbgs_per<double, DIM><<<prb_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, kappa, colour, x, b, z ? 1 : 0);
        }
        LAUNCH_CHECK(ctx);
      }
    }
    zero = false;
  }
  return ISDC_OK;
}

template <int DIM>
isdc_status vcycle_per(isdc_ctx* ctx, int slot, double a, double* x0, const double* b0) {
  Hier<double>& H = ctx->h64;
  double* xcur[kMaxLevels];
  isdc_status st;
  for (int l = 0; l < H.lb; ++l) {
    double* home = l == 0 ? x0 : H.x[l];
    double* x = home;
    const double* b = l == 0 ? b0 : H.b[l];
    bool zero = l > 0;
    const int s = H.side[l], sc = H.side[l + 1];
    if (ctx->opt.nu1 == 0 && zero) {
      CUDA_TRY(ctx, cudaMemsetAsync(x, 0, H.npts[l] * sizeof(double), ctx->stream));
      zero = false;
    }
    if ((st = smooth_level_per<DIM>(ctx, H, l, a, x, home, b, zero, ctx->opt.nu1)) != ISDC_OK) return st;
    const LevelCoef lf = coef_per(DIM, s, a);
    const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
    {
      ProfScope ps(ctx, l == 0 ? PC_RESIDUAL0 : PC_RESIDUALC, 3.0 * Np * 8, (nb_ops(DIM) + 2.0) * Np, true);
      k_residual_per<double, DIM><<<pp_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, lf.kappa, x, b, H.r[l]);
    }
    LAUNCH_CHECK(ctx);
    {
      const double ws = lf.d / (coef_per(DIM, sc, a).d * (DIM == 2 ? 16.0 : 64.0));
      ProfScope ps(ctx, l == 0 ? PC_RESTRICT0 : PC_RESTRICTC, (Np + Nc) * 8, (DIM == 2 ? 9.0 : 27.0) * Nc, true);
      k_restrict_per<double, DIM><<<pp_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
    }
    LAUNCH_CHECK(ctx);
    xcur[l] = x;
  }
  {  // the levels with side <= 32 (2D) / 8 (3D) in one block, the side-4 one by the dense inverse
    BottomParamsPer B{};
    B.nlev = H.nlev - H.lb;
    for (int q = 0; q < B.nlev; ++q) {
      const int s = H.side[H.lb + q];
      const LevelCoef lf = coef_per(DIM, s, a);
      B.side[q] = s;
      B.kappa[q] = lf.kappa;
      B.rscale[q] = q + 1 < B.nlev ? lf.d / (coef_per(DIM, H.side[H.lb + q + 1], a).d * (DIM == 2 ? 16.0 : 64.0)) : 0.0;
    }
    B.smoother = ctx->opt.smoother;
    B.nu1 = ctx->opt.nu1;
    B.nu2 = ctx->opt.nu2;
    B.omega = ctx->opt.omega;
    B.G = H.Ainv + size_t(slot) * ainv_slot(ctx);
    const double* bb = H.lb == 0 ? b0 : H.b[H.lb];
    double* xb = H.lb == 0 ? x0 : H.x[H.lb];
    ProfScope ps(ctx, PC_BOTTOM, 2.0 * double(H.npts[H.lb]) * 8, 0.0, true);
    k_bottom_per<DIM><<<1, kBottomThreads, H.bottom_smem, ctx->stream>>>(B, bb, xb, H.lb == 0 ? 1 : 0);
    LAUNCH_CHECK(ctx);
    xcur[H.lb] = xb;
  }
  for (int l = H.lb - 1; l >= 0; --l) {
    const int s = H.side[l], sc = H.side[l + 1];
    double* home = l == 0 ? x0 : H.x[l];
    double* x = xcur[l];
    {
      const double Np = double(H.npts[l]), Nc = double(H.npts[l + 1]);
      ProfScope ps(ctx, l == 0 ? PC_PROLONG0 : PC_PROLONGC, (2.0 * Np + Nc) * 8, (DIM == 2 ? 6.0 : 10.0) * Np, true);
      k_prolong_per<double, DIM><<<pp_grid(DIM, s), kBlock, 0, ctx->stream>>>(sc, xcur[l + 1], x);
    }
    LAUNCH_CHECK(ctx);
    bool zero = false;
    if ((st = smooth_level_per<DIM>(ctx, H, l, a, x, home, l == 0 ? b0 : H.b[l], zero, ctx->opt.nu2)) != ISDC_OK)
      return st;
    xcur[l] = x;
  }
  if (xcur[0] != x0)
    CUDA_TRY(ctx, cudaMemcpyAsync(x0, xcur[0], H.npts[0] * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  return ISDC_OK;
}

template <int DIM>
isdc_status node_residual_norm_per(isdc_ctx* ctx, double a, const double* x, const double* b, double* out) {
  const int s = ctx->n;
  const LevelCoef lf = coef_per(DIM, s, a);
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal + 1, 0, sizeof(unsigned long long), ctx->stream));
  {
    ProfScope ps(ctx, PC_RESNORM, 16.0 * double(ctx->N), (nb_ops(DIM) + 3.0) * double(ctx->N), true);
    k_resnorm_per<DIM><<<pp_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, lf.kappa, lf.d, x, b, ctx->d_scal + 1);
  }
  LAUNCH_CHECK(ctx);
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scal + 1, ctx->d_scal + 1, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned long long bits = ctx->h_scal[1];
  std::memcpy(out, &bits, sizeof(double));
  return ISDC_OK;
}

template <int DIM, int OFF, int P>
void launch_sweep_end_b_p(isdc_ctx* ctx) {
  const double nu_h2 = ctx->nu / (ctx->h * ctx->h), inv_h = 1.0 / ctx->h;
  k_sweep_end_b<DIM, OFF, P><<<pp_grid(DIM, ctx->n), kBlock, 0, ctx->stream>>>(
      ctx->n, ctx->N, nu_h2, inv_h, ctx->tables, ctx->U, ctx->F, ctx->FE, ctx->C, ctx->d_scal);
}

// End of a Burgers sweep: f and f^E at the last point, SDC residual, next C_m.
template <int DIM>
isdc_status sweep_end_b(isdc_ctx* ctx) {
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_scal, 0, sizeof(unsigned long long), ctx->stream));
  {
    const double M = ctx->M, P = ctx->P, Np = double(ctx->N);
    // algorithmic FP64 operations: WENO5 advection kWenoOps per axis (one face
    // flux per point and axis), Laplacian, dt Q f, residual, C_m
    ProfScope ps(ctx, PC_SWEEP_END, (2.0 * P + 2.0 * (P - 1.0) + 2.0 + (P - 1.0)) * 8.0 * Np,
                 (DIM * kWenoOps + nb_ops(DIM) + 3.0 + (P - 1.0) * M + 6.0 * (P - 1.0) - 1.0) * Np, true);
    if (ctx->off) {
      switch (ctx->P) {
        case 3: launch_sweep_end_b_p<DIM, 1, 3>(ctx); break;
        case 4: launch_sweep_end_b_p<DIM, 1, 4>(ctx); break;
        case 5: launch_sweep_end_b_p<DIM, 1, 5>(ctx); break;
        case 6: launch_sweep_end_b_p<DIM, 1, 6>(ctx); break;
        case 7: launch_sweep_end_b_p<DIM, 1, 7>(ctx); break;
        default: launch_sweep_end_b_p<DIM, 1, 8>(ctx); break;
      }
    } else {
      switch (ctx->P) {
        case 2: launch_sweep_end_b_p<DIM, 0, 2>(ctx); break;
        case 3: launch_sweep_end_b_p<DIM, 0, 3>(ctx); break;
        case 4: launch_sweep_end_b_p<DIM, 0, 4>(ctx); break;
        case 5: launch_sweep_end_b_p<DIM, 0, 5>(ctx); break;
        case 6: launch_sweep_end_b_p<DIM, 0, 6>(ctx); break;
        default: launch_sweep_end_b_p<DIM, 0, 7>(ctx); break;
      }
    }
  }
  LAUNCH_CHECK(ctx);
  return ISDC_OK;
}

// One Burgers sweep (Sec. 2, Eq. 4 with f^E the WENO5 advection).
template <int DIM>
isdc_status sweep_once_b(isdc_ctx* ctx, int n_vcycles, long long* vcycles) {
  const int n = ctx->n, P = ctx->P;
  const size_t N = ctx->N;
  const double nu_h2 = ctx->nu / (ctx->h * ctx->h), inv_h = 1.0 / ctx->h;
  isdc_status st;
  for (int m = 0; m < P - 1; ++m) {
    const double dtm = ctx->tables.dtm[m], a = dtm * ctx->nu;
    const double inv_d0 = 1.0 / coef_per(DIM, n, a).d;
    {
      ProfScope ps(ctx, PC_RHS, (m >= 1 ? 5.0 : 4.0) * 8.0 * double(N),
                   (m >= 1 ? DIM * kWenoOps + nb_ops(DIM) + 6.0 : 4.0) * double(N), true);
      k_rhs_b<DIM><<<pp_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, nu_h2, inv_h, dtm, inv_d0, ctx->U + m * N,
                                                                ctx->C + m * N, ctx->b, ctx->F + m * N,
                                                                ctx->FE + m * N, m >= 1 ? 1 : 0);
    }
    LAUNCH_CHECK(ctx);
    double* x = ctx->U + (m + 1) * N;  // initial guess u_{m+1}^k (Sec. 4.3)
    if (n_vcycles > 0 && !ctx->opt.vcycle_cap) {
      for (int c = 0; c < n_vcycles; ++c)
        if ((st = vcycle_per<DIM>(ctx, m, a, x, ctx->b)) != ISDC_OK) return st;
      *vcycles += n_vcycles;
    } else {
      const int limit = n_vcycles > 0 ? n_vcycles : ctx->opt.mg_max_cycles;
      for (int c = 0; c < limit; ++c) {
        double rn;
        if ((st = node_residual_norm_per<DIM>(ctx, a, x, ctx->b, &rn)) != ISDC_OK) return st;
        if (!(rn > ctx->opt.mg_tol)) break;
        if ((st = vcycle_per<DIM>(ctx, m, a, x, ctx->b)) != ISDC_OK) return st;
        ++*vcycles;
      }
    }
  }
  return sweep_end_b<DIM>(ctx);
}

// One SDC sweep with the compact stencil (Sec. 3, Eq. 5): the right-hand
// sides carry W, the node solves invert W - dt_m nu L_9 (FP64 V-cycles).
isdc_status sweep_once9(isdc_ctx* ctx, int n_vcycles, long long* vcycles) {
  const int n = ctx->n, P = ctx->P;
  const size_t N = ctx->N;
  const double nu6 = ctx->nu / (6.0 * ctx->h * ctx->h);
  isdc_status st;
  for (int m = 0; m < P - 1; ++m) {
    const double dtm = ctx->tables.dtm[m], a = dtm * ctx->nu;
    const Coef9 k = coef9(n, a);
    {
      ProfScope ps(ctx, PC_RHS, (m >= 1 ? 5.0 : 3.0) * 8.0 * double(N), (m >= 1 ? 40.0 : 12.0) * double(N), true);
      k_rhs9<<<pt_grid(2, n), kBlock, 0, ctx->stream>>>(n, nu6, ctx->opt.reaction, dtm, 1.0 / k.c0, ctx->U + m * N,
                                                        ctx->C + m * N, ctx->b, m >= 1 ? ctx->F + m * N : nullptr,
                                                        m >= 1 ? ctx->G + m * N : nullptr);
    }
    LAUNCH_CHECK(ctx);
    double* x = ctx->U + (m + 1) * N;  // initial guess u_{m+1}^k (Sec. 4.3)
    if (n_vcycles > 0 && !ctx->opt.vcycle_cap) {
      for (int c = 0; c < n_vcycles; ++c)
        if ((st = vcycle9(ctx, m, a, x, ctx->b)) != ISDC_OK) return st;
      *vcycles += n_vcycles;
    } else {  // classical SDC, or L as a cap, with the node residual test
      const int limit = n_vcycles > 0 ? n_vcycles : ctx->opt.mg_max_cycles;
      for (int c = 0; c < limit; ++c) {
        double rn;
        if ((st = node_residual_norm9(ctx, a, x, ctx->b, &rn)) != ISDC_OK) return st;
        if (!(rn > ctx->opt.mg_tol)) break;
        if ((st = vcycle9(ctx, m, a, x, ctx->b)) != ISDC_OK) return st;
        ++*vcycles;
      }
    }
  }
  return sweep_end9(ctx);
}

// One SDC sweep (Sec. 2, Eq. 4): the P-1 node solves (M-1 for Gauss-Lobatto,
// M otherwise) and the sweep end (f at the last point, SDC residual, next C_m).
// *vcycles accumulates the V-cycles spent.
template <int DIM>
isdc_status sweep_once(isdc_ctx* ctx, int n_vcycles, long long* vcycles) {
  if (ctx->stencil == 1) return sweep_once9(ctx, n_vcycles, vcycles);
  if (ctx->equation == 1) return sweep_once_b<DIM>(ctx, n_vcycles, vcycles);
  const int n = ctx->n, P = ctx->P;
  const size_t N = ctx->N;
  const double nu_h2 = ctx->nu / (ctx->h * ctx->h);
  isdc_status st;
  for (int m = 0; m < P - 1; ++m) {
    const double dtm = ctx->tables.dtm[m];
    const double inv_d0 = 1.0 / level_coef(DIM, n, dtm * ctx->nu).d;
    double* x = ctx->U + (m + 1) * N;  // initial guess u_{m+1}^k (Sec. 4.3)
    const double a = dtm * ctx->nu;
    if (ctx->cprime) {  // FP32 V-cycles, fixed count: rhs and defect in one pass
      {
        ProfScope ps(ctx, PC_RHS, (m >= 1 ? 36.0 : 20.0) * double(N), (m >= 1 ? nb_ops(DIM) + 7.0 : 5.0) * double(N),
                     true);
        double* Fm = m >= 1 ? ctx->F + m * N : nullptr;
        double* FEm = ctx->FE + m * N;
        if (ctx->sp_x)
          k_rhs_defect_split<DIM><<<rb_grid(DIM, n), kBlock, 0, ctx->stream>>>(
              n, nu_h2, ctx->opt.reaction, dtm, inv_d0, ctx->U + m * N, ctx->C + m * N, Fm, FEm, ctx->sp_b,
              ctx->sp_b + ctx->hn);
        else
          k_rhs_defect<DIM><<<pt_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, nu_h2, ctx->opt.reaction, dtm, inv_d0,
                                                                         ctx->U + m * N, ctx->C + m * N, Fm, FEm,
                                                                         ctx->h32.b[0]);
      }
      LAUNCH_CHECK(ctx);
      if ((st = node_solve<DIM>(ctx, m, a, x, nullptr, n_vcycles, true)) != ISDC_OK) return st;
      *vcycles += n_vcycles;
      continue;
    }
    {
      ProfScope ps(ctx, PC_RHS, (m >= 1 ? 5.0 : 3.0) * 8.0 * double(N),
                   (m >= 1 ? nb_ops(DIM) + 7.0 : 5.0) * double(N), true);
      k_rhs<DIM><<<pt_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, nu_h2, ctx->opt.reaction, dtm, inv_d0,
                                                              ctx->U + m * N, ctx->C + m * N, ctx->b,
                                                              m >= 1 ? ctx->F + m * N : nullptr, ctx->FE + m * N);
    }
    LAUNCH_CHECK(ctx);
    if (n_vcycles > 0 && !ctx->opt.vcycle_cap) {
      if ((st = node_solve<DIM>(ctx, m, a, x, ctx->b, n_vcycles)) != ISDC_OK) return st;
      *vcycles += n_vcycles;
    } else {  // classical SDC: multigrid to a tolerance (Sec. 3); or L as a cap with that early exit
      const int limit = n_vcycles > 0 ? n_vcycles : ctx->opt.mg_max_cycles;
      for (int c = 0; c < limit; ++c) {
        double rn;
        if ((st = node_residual_norm<DIM>(ctx, a, x, ctx->b, &rn)) != ISDC_OK) return st;
        if (!(rn > ctx->opt.mg_tol)) break;
        if ((st = node_solve<DIM>(ctx, m, a, x, ctx->b, 1)) != ISDC_OK) return st;
        ++*vcycles;
      }
    }
  }
  return sweep_end<DIM>(ctx);
}

// Capture one sweep as a CUDA graph (on a private stream, so that the caller
// may run on the legacy default stream); the graph also copies the residual
// bits to the pinned host scalar.
template <int DIM>
isdc_status capture_sweep(isdc_ctx* ctx, int n_vcycles) {
  Profiler& P = ctx->prof;
  const unsigned mask = P.on ? P.event_mask : 0u;
  if (ctx->sweep_graph && ctx->graph_vcycles == n_vcycles && ctx->graph_mask == mask &&
      ctx->graph_counted == P.on) {
    return ISDC_OK;
  }
  if (ctx->sweep_graph) {
    cudaGraphExecDestroy(ctx->sweep_graph);
    ctx->sweep_graph = nullptr;
  }
  if (!ctx->cap_stream) CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  P.capturing = P.on;
  P.gused = 0;
  for (int c = 0; c < PC_COUNT; ++c) {
    P.d_launches[c] = 0;
    P.d_bytes[c] = P.d_dp[c] = P.d_sp[c] = 0.0;
  }
  long long dummy = 0;
  isdc_status st = sweep_once<DIM>(ctx, n_vcycles, &dummy);
  P.capturing = false;
  if (st == ISDC_OK) {
    cudaError_t e = cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e != cudaSuccess) st = fail(ctx, ISDC_ERR_CUDA, "capture copy: %s", cudaGetErrorString(e));
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->stream = user;
  if (st != ISDC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(ctx, ISDC_ERR_CUDA, "sweep capture: %s", cudaGetErrorString(e));
  if (ctx->opt.use_graphs == 1 && (e = host::programmatic_edges(g)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(ctx, ISDC_ERR_CUDA, "sweep graph edges: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&ctx->sweep_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, ISDC_ERR_CUDA, "sweep graph: %s", cudaGetErrorString(e));
  ctx->graph_vcycles = n_vcycles;
  ctx->graph_mask = mask;
  ctx->graph_counted = P.on;
  return ISDC_OK;
}

template <int DIM>
isdc_status run_step(isdc_ctx* ctx, double* u, int n_sweeps, int n_vcycles) {
  const int n = ctx->n, P = ctx->P;
  const size_t N = ctx->N;
  const double nu_h2 = ctx->nu / (ctx->h * ctx->h);
  isdc_status st;
  const double nu6 = ctx->nu / (6.0 * ctx->h * ctx->h);
  if (ctx->nodes_pending && ctx->stencil == 1) {
    // resume with the compact stencil: f~ and nu L_9 u at t_0 and every node
    if (ctx->off)
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->U, u, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    for (int m = 0; m < P; ++m) {
      {
        ProfScope ps(ctx, PC_EVAL_F, 24.0 * double(N), 30.0 * double(N), true);
        k_eval_f9<<<pt_grid(2, n), kBlock, 0, ctx->stream>>>(n, nu6, ctx->opt.reaction, ctx->U + m * N,
                                                             ctx->F + m * N, ctx->G + m * N);
      }
      LAUNCH_CHECK(ctx);
    }
    ctx->nodes_pending = 0;
  } else if (ctx->stencil == 1) {
    {
      ProfScope ps(ctx, PC_SPREAD, (1.0 + 3.0 * P) * 8.0 * double(N), 30.0 * double(N), true);
      k_spread9<<<pt_grid(2, n), kBlock, 0, ctx->stream>>>(n, N, nu6, ctx->opt.reaction, P, u, ctx->U, ctx->F,
                                                           ctx->G);
    }
    LAUNCH_CHECK(ctx);
  } else if (ctx->equation == 1) {
    const double inv_h = 1.0 / ctx->h;
    if (ctx->nodes_pending) {  // resume: f and f^E at t_0 and every node
      if (ctx->off)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->U, u, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      for (int m = 0; m < P; ++m) {
        {
          ProfScope ps(ctx, PC_EVAL_F, 24.0 * double(N), (DIM * kWenoOps + nb_ops(DIM) + 3.0) * double(N), true);
          k_eval_f_b<DIM><<<pp_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, nu_h2, inv_h, ctx->U + m * N,
                                                                       ctx->F + m * N, ctx->FE + m * N);
        }
        LAUNCH_CHECK(ctx);
      }
      ctx->nodes_pending = 0;
    } else {
      {
        ProfScope ps(ctx, PC_SPREAD, (1.0 + 3.0 * P) * 8.0 * double(N), (DIM * kWenoOps + nb_ops(DIM) + 3.0) * double(N),
                     true);
        k_spread_b<DIM><<<pp_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, N, nu_h2, inv_h, P, u, ctx->U, ctx->F,
                                                                     ctx->FE);
      }
      LAUNCH_CHECK(ctx);
    }
  } else if (ctx->nodes_pending) {
    // resume: the nodes were set; t_0 (not a node unless Gauss-Lobatto) is u
    if (ctx->off)
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->U, u, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    for (int m = 0; m < P; ++m) {  // f^E of t_0 too (the first C needs it)
      {
        ProfScope ps(ctx, PC_EVAL_F, 24.0 * double(N), (nb_ops(DIM) + 5.0) * double(N), true);
        k_eval_f<DIM><<<pt_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, nu_h2, ctx->opt.reaction, ctx->U + m * N,
                                                                   ctx->F + m * N, ctx->FE + m * N);
      }
      LAUNCH_CHECK(ctx);
    }
    ctx->nodes_pending = 0;
  } else {
    {
      ProfScope ps(ctx, PC_SPREAD, (1.0 + 3.0 * P) * 8.0 * double(N), (nb_ops(DIM) + 5.0) * double(N), true);
      k_spread<DIM><<<pt_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, N, nu_h2, ctx->opt.reaction, P, u, ctx->U,
                                                                 ctx->F, ctx->FE);
    }
    LAUNCH_CHECK(ctx);
  }
  ctx->cprime = ctx->opt.vcycle_fp32 && n_vcycles > 0 && !ctx->opt.vcycle_cap;
  // C_m of the first sweep
  if ((st = ctx->stencil == 1 ? sweep_end9(ctx) : ctx->equation == 1 ? sweep_end_b<DIM>(ctx) : sweep_end<DIM>(ctx)) !=
      ISDC_OK)
    return st;

  const bool until_tol = n_sweeps <= 0;
  const int cap = until_tol ? ctx->opt.max_sweeps : n_sweeps;
  long long vcycles = 0;
  int k = 0;
  isdc_status result = ISDC_OK;
  ctx->hist_count = 0;
  // sweeps with a fixed V-cycle count replay one captured graph (unless the
  // profiler or a per-sweep history copy needs the launches one by one)
  const bool graph = ctx->opt.use_graphs && n_vcycles > 0 && !ctx->opt.vcycle_cap &&
                     (until_tol || !ctx->record_history);
  if (graph && (st = capture_sweep<DIM>(ctx, n_vcycles)) != ISDC_OK) return st;
  for (;;) {
    if (graph) {
      CUDA_TRY(ctx, cudaGraphLaunch(ctx->sweep_graph, ctx->stream));
      vcycles += (long long)n_vcycles * (P - 1);
      if (ctx->prof.on) {  // read the replay's event nodes before the next replay re-records them
        if (ctx->prof.event_mask) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        prof_graph_replayed(ctx);
      }
    } else if ((st = sweep_once<DIM>(ctx, n_vcycles, &vcycles)) != ISDC_OK) {
      return st;
    }
    ++k;
    if (!graph && (until_tol || ctx->record_history)) {
      if (k - 1 < ctx->hist_cap)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_hist + (k - 1), ctx->d_scal, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, ctx->stream));
      ctx->hist_count = std::min(k, ctx->hist_cap);
    }
    if (until_tol) {
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (graph) {
        if (k - 1 < ctx->hist_cap) ctx->h_hist[k - 1] = ctx->h_scal[0];
        ctx->hist_count = std::min(k, ctx->hist_cap);
      }
      const double R = bits_to_double(ctx->h_hist[k - 1]);
      if (!std::isfinite(R)) { result = fail(ctx, ISDC_ERR_NONFINITE, "SDC residual is %g after sweep %d", R, k); break; }
      if (R < ctx->opt.tol) break;
      if (k >= cap) {
        result = fail(ctx, ISDC_ERR_NOT_CONVERGED, "SDC residual %g >= tol %g after %d sweeps", R, ctx->opt.tol, k);
        break;
      }
    } else if (k >= cap) {
      break;
    }
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                ctx->stream));
  if (ctx->node_kind == ISDC_NODES_GAUSS_LEGENDRE && ctx->stencil == 1) {
    // the same with f = f^E + W^{-1} nu L_9 u: u = u_0 + dt sum w f^E + W^{-1} (dt sum w nu L_9 u)
    {
      ProfScope ps(ctx, PC_SPREAD, (ctx->M + 1.0) * 8.0 * double(N), 2.0 * ctx->M * double(N), true);
      k_gauss_end9_sum<<<pt_grid(2, n), kBlock, 0, ctx->stream>>>(n, N, ctx->ends, ctx->G, ctx->b);
    }
    LAUNCH_CHECK(ctx);
    const double* wy = nullptr;
    if ((st = w_inverse(ctx, 1, ctx->b, ctx->Rs, ctx->Rs + N, kWinvEndIters, &wy)) != ISDC_OK) return st;
    {
      ProfScope ps(ctx, PC_SPREAD, (ctx->M + 3.0) * 8.0 * double(N), 4.0 * ctx->M * double(N), true);
      k_gauss_end9<<<pt_grid(2, n), kBlock, 0, ctx->stream>>>(n, N, ctx->ends, ctx->opt.reaction, ctx->U, wy, u);
    }
  } else if (ctx->node_kind == ISDC_NODES_GAUSS_LEGENDRE) {
    // tau_M < 1: the step ends with the full-step quadrature of the collocation rule
    ProfScope ps(ctx, PC_SPREAD, (ctx->M + 2.0) * 8.0 * double(N), 2.0 * ctx->M * double(N), true);
    k_gauss_end<DIM><<<pt_grid(DIM, n), kBlock, 0, ctx->stream>>>(n, N, ctx->ends, ctx->U, ctx->F, u);
  } else {
    CUDA_TRY(ctx, cudaMemcpyAsync(u, ctx->U + (P - 1) * N, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  }
  LAUNCH_CHECK(ctx);
  ctx->last_sweeps = k;
  ctx->last_vcycles = vcycles;
  return result;
}

// Autotuner for the red-black smoothers (3D): on every grid-wide level with
// side >= 31, time red and black passes with 1 to 32 points per thread along
// a diagonal, streamed or in one burst (natural layout; 1, 2, 4 or 8 z-planes
// on the split level) on the context's own arrays of that level (zeroed
// first; the values do not change the timing) and keep the fastest.  Runs
// once, in isdc_create.
template <typename T>
float time_rbgs_pass(isdc_ctx* ctx, int s, int zb, T* x, const T* b, float* xs0, float* bs0, size_t hn,
                     cudaEvent_t e0, cudaEvent_t e1, isdc_status* st, int pairs) {
  *st = ISDC_OK;
  if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { *st = ISDC_ERR_CUDA; return 0.f; }
  for (int c2 = 0; c2 < 2 * pairs; ++c2) {
    const int colour = c2 & 1;
    if (xs0) {
      launch_rbgs_split<3>(ctx->stream, zb, s, 0.1f, colour, xs0 + colour * hn, xs0 + (1 - colour) * hn,
                           bs0 + colour * hn, false);
    } else {
      launch_rbgs<T, 3>(ctx->stream, s, T(0.1), colour, x, b, false, zb);
    }
  }
  float ms = 0.f;
  if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    *st = fail(ctx, ISDC_ERR_CUDA, "smoother autotuning failed");
  return ms;
}

template <typename T>
isdc_status tune_levels(isdc_ctx* ctx, Hier<T>& H, T* x0, T* b0, bool split0, cudaEvent_t e0, cudaEvent_t e1) {
  // natural layout: diagonal runs streamed (2..32 points) or in one burst
  // (1..8, negative); split FP32 level: 1..8 z-planes
  const int cand[9] = {-1, -2, -4, -8, 2, 4, 8, 16, 32};
  const int split_cand[4] = {1, 2, 4, 8};
  for (int l = 0; l < H.lb; ++l) {
    const int s = H.side[l];
    if (s < 31) break;
    T* x = l == 0 ? x0 : H.x[l];
    T* b = l == 0 ? b0 : H.b[l];
    const bool split = l == 0 && split0;
    if (!split && ctx->opt.rb_run != 0) {  // fixed by the caller
      ctx->zbl[l] = ctx->opt.rb_run;
      if (l == 0) (sizeof(T) == 8 ? ctx->zb64 : ctx->zb32) = ctx->opt.rb_run < 0 ? -ctx->opt.rb_run : ctx->opt.rb_run;
      continue;
    }
    if (split) {
      CUDA_TRY(ctx, cudaMemsetAsync(ctx->sp_x, 0, 2 * ctx->hn * sizeof(float), ctx->stream));
      CUDA_TRY(ctx, cudaMemsetAsync(ctx->sp_b, 0, 2 * ctx->hn * sizeof(float), ctx->stream));
    } else {
      CUDA_TRY(ctx, cudaMemsetAsync(x, 0, H.npts[l] * sizeof(T), ctx->stream));
      CUDA_TRY(ctx, cudaMemsetAsync(b, 0, H.npts[l] * sizeof(T), ctx->stream));
    }
    float best = 1e30f;
    int best_zb = 1;
    // small levels take a few microseconds a pass: time 16 red-black pairs per
    // trial there (2 above 1M points) and keep each form's best of two rounds
    const int pairs = H.npts[l] >= (size_t(1) << 20) ? 2 : 16;
    for (int rep = 0; rep < 3; ++rep)  // the first round warms up
      for (int c = 0; c < (split ? 4 : 9); ++c) {
        isdc_status st;
        const int zb = split ? split_cand[c] : cand[c];
        const float ms = time_rbgs_pass<T>(ctx, s, zb, x, b, split ? ctx->sp_x : nullptr,
                                           split ? ctx->sp_b : nullptr, ctx->hn, e0, e1, &st, pairs);
        if (st != ISDC_OK) return st;
        if (rep >= 1 && ms < best) {
          best = ms;
          best_zb = zb;
        }
      }
    if (split) ctx->zb32 = best_zb;
    else ctx->zbl[l] = best_zb;
    if (l == 0 && !split) (sizeof(T) == 8 ? ctx->zb64 : ctx->zb32) = best_zb < 0 ? -best_zb : best_zb;
  }
  return ISDC_OK;
}

// Temporal blocking of the split FP32 fine level (3D): time max(nu1, nu2)
// red-black sweeps as separate colour passes (with the planes per thread just
// chosen) and as blocked passes of 1 and 2 sweeps with 16, 32, 64 and 128
// planes per block, on the context's own arrays; keep the fastest.
isdc_status tune_blocking(isdc_ctx* ctx, cudaEvent_t e0, cudaEvent_t e1) {
  struct Cand { int depth, zc; };
  const Cand cand[9] = {{0, 32}, {1, 16}, {1, 32}, {1, 64}, {1, 128}, {2, 16}, {2, 32}, {2, 64}, {2, 128}};
  const int nsw = std::max(ctx->opt.nu1, ctx->opt.nu2);
  float best = 1e30f;
  Cand pick = cand[0];
  for (int rep = 0; rep < 2; ++rep)  // the first round warms up
    for (const Cand& c : cand) {
      ctx->tb_depth = c.depth;
      ctx->tb_zc = c.zc;
      float* xb = ctx->sp_x + ctx->hn;
      CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
      isdc_status st = smooth_split<3>(ctx, 0.1f, nsw, false, &xb);
      if (st != ISDC_OK) return st;
      CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
      CUDA_TRY(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1 && ms < best) {
        best = ms;
        pick = c;
      }
    }
  ctx->tb_depth = pick.depth;
  ctx->tb_zc = pick.zc;
  return ISDC_OK;
}

// Residual + restriction of every grid-wide level: the two-launch form and the
// fused launch (3D: 4, 8 or 16 coarse planes per block) give the same values
// bit for bit; time each on the level's own arrays and keep the fastest.
template <typename T, int DIM>
isdc_status time_transfer(isdc_ctx* ctx, Hier<T>& H, int l, const T* x, const T* b, bool split, int kc, int reps,
                          cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  const int s = H.side[l], sc = H.side[l + 1];
  const T kappa = T(0.1), ws = T(0.01);
  const bool red_only = ctx->opt.smoother == ISDC_SMOOTHER_RBGS && ctx->opt.nu1 >= 1;
  const dim3 gf = resrestrict_grid(DIM, sc, kc), bf(kRrTX, kRrTY, 1);
  CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
  for (int r = 0; r < reps; ++r) {
    if (split) {
      const size_t hn = ctx->hn;
      const float *xr = ctx->sp_x, *xb = ctx->sp_x + hn, *br = ctx->sp_b;
      if (kc > 0) {
        k_resrestrict_red_split<DIM><<<gf, bf, 0, ctx->stream>>>(sc, float(kappa), float(ws), xr, xb, br,
                                                                 reinterpret_cast<float*>(H.b[1]), kc);
      } else {
        k_residual_red_split<DIM><<<rb_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, float(kappa), xr, xb, br,
                                                                               ctx->sp_r);
        k_restrict_red_split<DIM><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, float(ws), ctx->sp_r,
                                                                                reinterpret_cast<float*>(H.b[1]));
      }
    } else if (kc > 0) {
      if (red_only) k_resrestrict<T, DIM, true><<<gf, bf, 0, ctx->stream>>>(sc, kappa, ws, x, b, H.b[l + 1], kc);
      else k_resrestrict<T, DIM, false><<<gf, bf, 0, ctx->stream>>>(sc, kappa, ws, x, b, H.b[l + 1], kc);
    } else if (red_only) {
      k_residual<T, DIM, true><<<rb_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, kappa, x, b, H.r[l]);
      k_restrict<T, DIM, true><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
    } else {
      k_residual<T, DIM, false><<<pt_grid(DIM, s), kBlock, 0, ctx->stream>>>(s, kappa, x, b, H.r[l]);
      k_restrict<T, DIM, false><<<pt_grid(DIM, sc), kBlock, 0, ctx->stream>>>(sc, ws, H.r[l], H.b[l + 1]);
    }
  }
  CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
  CUDA_TRY(ctx, cudaEventSynchronize(e1));
  CUDA_TRY(ctx, cudaGetLastError());
  CUDA_TRY(ctx, cudaEventElapsedTime(ms, e0, e1));
  return ISDC_OK;
}

template <typename T, int DIM>
isdc_status tune_transfer(isdc_ctx* ctx, Hier<T>& H, T* x0, T* b0, bool split0, cudaEvent_t e0, cudaEvent_t e1) {
  int* rr = sizeof(T) == 8 ? ctx->rr64 : ctx->rr32;
  const int cand3[4] = {0, 4, 8, 16}, cand2[2] = {0, 1};
  int dev = 0, sms = 0;
  CUDA_TRY(ctx, cudaGetDevice(&dev));
  CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int l = 0; l < H.lb; ++l) {
    const bool split = l == 0 && split0;
    T* x = l == 0 ? x0 : H.x[l];
    T* b = l == 0 ? b0 : H.b[l];
    if (split) {
      CUDA_TRY(ctx, cudaMemsetAsync(ctx->sp_x, 0, 2 * ctx->hn * sizeof(float), ctx->stream));
      CUDA_TRY(ctx, cudaMemsetAsync(ctx->sp_b, 0, 2 * ctx->hn * sizeof(float), ctx->stream));
    } else {
      CUDA_TRY(ctx, cudaMemsetAsync(x, 0, H.npts[l] * sizeof(T), ctx->stream));
      CUDA_TRY(ctx, cudaMemsetAsync(b, 0, H.npts[l] * sizeof(T), ctx->stream));
    }
    const int reps = H.npts[l] >= (size_t(1) << 20) ? 4 : 32;
    const int nc = DIM == 3 ? 4 : 2;
    float best = 1e30f;
    int pick = 0;
    for (int round = 0; round < 3; ++round)  // the first round warms up
      for (int c = 0; c < nc; ++c) {
        const int kc = DIM == 3 ? cand3[c] : cand2[c];
        if (kc > 0) {
          // a fused launch with fewer than two blocks per SM loses to the two
          // launches inside the replayed sweep (measured on the 127^2 workload:
          // 181.7 against 160 us per sweep) while winning a back-to-back timing
          // loop, so it is not a candidate there
          const dim3 gf = resrestrict_grid(DIM, H.side[l + 1], kc);
          if (size_t(gf.x) * gf.y * gf.z < size_t(2) * sms) continue;
        }
        float ms = 0.f;
        isdc_status st = time_transfer<T, DIM>(ctx, H, l, x, b, split, kc, reps, e0, e1, &ms);
        if (st != ISDC_OK) return st;
        if (round >= 1 && ms < best) {
          best = ms;
          pick = kc;
        }
      }
    if (split) ctx->rr_split = pick;
    else rr[l] = pick;
  }
  return ISDC_OK;
}

// Fixed forms (option fused_transfer 0 or 1) or the tuned choice (-1).
isdc_status setup_transfer(isdc_ctx* ctx) {
  if (ctx->stencil == 1 || ctx->equation == 1) return ISDC_OK;  // their own transfer kernels
  const int f = ctx->opt.fused_transfer;
  const bool fp32 = ctx->opt.vcycle_fp32 != 0;
  const int lb = fp32 ? ctx->h32.lb : ctx->h64.lb;
  for (int l = 0; l < lb; ++l) {
    const int sc = fp32 ? ctx->h32.side[l + 1] : ctx->h64.side[l + 1];
    const int kc = f == 1 ? (ctx->dim == 3 ? resrestrict_kc(sc) : 1) : 0;
    (fp32 ? ctx->rr32 : ctx->rr64)[l] = kc;
  }
  if (ctx->sp_x) ctx->rr_split = f == 1 ? (ctx->dim == 3 ? resrestrict_kc(ctx->h32.side[1]) : 1) : 0;
  if (f != -1) return ISDC_OK;
  cudaEvent_t e0, e1;
  CUDA_TRY(ctx, cudaEventCreate(&e0));
  CUDA_TRY(ctx, cudaEventCreate(&e1));
  isdc_status st;
  if (fp32)
    st = ctx->dim == 2 ? tune_transfer<float, 2>(ctx, ctx->h32, ctx->h32.x[0], ctx->h32.b[0], ctx->sp_x != nullptr, e0, e1)
                       : tune_transfer<float, 3>(ctx, ctx->h32, ctx->h32.x[0], ctx->h32.b[0], ctx->sp_x != nullptr, e0, e1);
  else
    st = ctx->dim == 2 ? tune_transfer<double, 2>(ctx, ctx->h64, ctx->U, ctx->b, false, e0, e1)
                       : tune_transfer<double, 3>(ctx, ctx->h64, ctx->U, ctx->b, false, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

isdc_status tune_smoother(isdc_ctx* ctx) {
  if (ctx->dim != 3 || ctx->opt.smoother != ISDC_SMOOTHER_RBGS) return ISDC_OK;
  cudaEvent_t e0, e1;
  CUDA_TRY(ctx, cudaEventCreate(&e0));
  CUDA_TRY(ctx, cudaEventCreate(&e1));
  isdc_status st = ctx->opt.vcycle_fp32
                       ? tune_levels<float>(ctx, ctx->h32, ctx->h32.x[0], ctx->h32.b[0], ctx->sp_x != nullptr, e0, e1)
                       : tune_levels<double>(ctx, ctx->h64, ctx->U, ctx->b, false, e0, e1);
  if (st == ISDC_OK && ctx->sp_xb) {
    if (ctx->opt.temporal_blocking >= 0) ctx->tb_depth = ctx->opt.temporal_blocking;
    else st = tune_blocking(ctx, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
ISDC_API isdc_status isdc_default_options(isdc_options* opt) {
  if (!opt) return ISDC_ERR_INVALID_ARG;
  opt->smoother = ISDC_SMOOTHER_JACOBI;
  opt->nu1 = 1;
  opt->nu2 = 1;
  opt->omega = 2.0 / 3.0;
  opt->vcycle_fp32 = 0;
  opt->reaction = ISDC_REACTION_ALLEN_CAHN;
  opt->tol = 1e-10;
  opt->max_sweeps = 100;
  opt->mg_tol = 1e-12;
  opt->mg_max_cycles = 50;
  opt->vcycle_cap = 0;
  opt->use_graphs = 1;
  opt->temporal_blocking = -1;
  opt->rb_run = 0;
  opt->fused_transfer = -1;
  opt->stencil = 0;
  opt->equation = 0;
  opt->stream = nullptr;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_collocation_tables(isdc_node_type nodes, int M, double* tau, double* Q, double* S) {
  if (nodes != ISDC_NODES_GAUSS_LOBATTO && nodes != ISDC_NODES_RADAU_RIGHT && nodes != ISDC_NODES_GAUSS_LEGENDRE) {
    snprintf(g_create_error, sizeof g_create_error, "unknown node type %d", int(nodes));
    return ISDC_ERR_INVALID_ARG;
  }
  if (M < 2 || M > kMaxM || !tau || !Q) {
    snprintf(g_create_error, sizeof g_create_error, "M must be in [2, %d] and tau, Q non-NULL", kMaxM);
    return ISDC_ERR_INVALID_ARG;
  }
  collocation_nodes(int(nodes), M, tau);
  q_matrix(M, tau, Q);
  if (S) {  // point to point: rows of Q, preceded by a zero row for t_0 unless t_0 is node 1
    const int off = nodes == ISDC_NODES_GAUSS_LOBATTO ? 0 : 1;
    for (int m = 0; m < M - 1 + off; ++m)
      for (int j = 0; j < M; ++j) {
        const double lo = m - off >= 0 ? Q[(m - off) * M + j] : 0.0;
        S[m * M + j] = Q[(m + 1 - off) * M + j] - lo;
      }
  }
  return ISDC_OK;
}

ISDC_API void isdc_destroy(isdc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->U);
  cudaFree(ctx->F);
  cudaFree(ctx->C);
  cudaFree(ctx->G);
  cudaFree(ctx->Rs);
  cudaFree(ctx->FE);
  cudaFree(ctx->b);
  cudaFree(ctx->u_dev);
  free_hier(ctx->h64, false);
  free_hier(ctx->h32, true);
  cudaFree(ctx->sp_x);
  cudaFree(ctx->sp_xb);
  cudaFree(ctx->sp_b);
  cudaFree(ctx->sp_r);
  cudaFree(ctx->d_scal);
  cudaFreeHost(ctx->h_scal);
  cudaFreeHost(ctx->h_hist);
  if (ctx->sweep_graph) cudaGraphExecDestroy(ctx->sweep_graph);
  for (auto& r : ctx->prof.gpool) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto& r : ctx->prof.pool) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

ISDC_API isdc_status isdc_create(int ndim, const int64_t* dims, double nu, isdc_node_type nodes, int M, double dt,
                                 const isdc_options* opt, isdc_ctx** out) {
  if (!out) return fail(nullptr, ISDC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(nullptr, ISDC_ERR_INVALID_ARG, "ndim must be 2 or 3 (got %d)", ndim);
  if (!dims) return fail(nullptr, ISDC_ERR_INVALID_ARG, "dims is NULL");
  const int64_t n = dims[0];
  for (int a = 1; a < ndim; ++a)
    if (dims[a] != n) return fail(nullptr, ISDC_ERR_UNSUPPORTED, "only equal sides are implemented");
  const int equation = opt ? opt->equation : 0;
  if (equation != 0 && equation != 1) return fail(nullptr, ISDC_ERR_INVALID_ARG, "unknown equation %d", equation);
  if (equation == 0 && (n < 3 || ((n + 1) & n) != 0))
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "side must be 2^j - 1 with j >= 2 (got %lld)", (long long)n);
  if (equation == 1 && (n < 8 || (n & (n - 1)) != 0))
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "periodic side must be 2^j with j >= 3 (got %lld)", (long long)n);
  if ((ndim == 2 && n > 46339) || (ndim == 3 && n > 1289))
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "grid too large for 32-bit point indices");
  {
    int nlev = 1;
    for (int64_t s = n; equation == 1 ? s > 4 : s > 3; s = equation == 1 ? s / 2 : (s - 1) / 2) ++nlev;
    if (nlev > kMaxLevels)
      return fail(nullptr, ISDC_ERR_INVALID_ARG, "side %lld needs %d multigrid levels (at most %d)", (long long)n, nlev,
                  kMaxLevels);
  }
  if (nodes != ISDC_NODES_GAUSS_LOBATTO && nodes != ISDC_NODES_RADAU_RIGHT && nodes != ISDC_NODES_GAUSS_LEGENDRE)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "unknown node type %d", int(nodes));
  if (M < 2 || M > kMaxM) return fail(nullptr, ISDC_ERR_INVALID_ARG, "M must be in [2, %d] (got %d)", kMaxM, M);
  if (!(nu > 0) || !std::isfinite(nu) || !(dt > 0) || !std::isfinite(dt))
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "nu and dt must be positive and finite");
  isdc_options o;
  if (opt) o = *opt; else isdc_default_options(&o);
  if (o.smoother != ISDC_SMOOTHER_JACOBI && o.smoother != ISDC_SMOOTHER_RBGS)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "unknown smoother %d", o.smoother);
  if (o.smoother == ISDC_SMOOTHER_JACOBI && !(o.omega > 0 && o.omega <= 1))
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "the Jacobi damping omega must be in (0, 1]");
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1 || o.nu1 > 16 || o.nu2 > 16)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "nu1, nu2 must be in [0, 16] with nu1 + nu2 >= 1");
  if (o.reaction != ISDC_REACTION_NONE && o.reaction != ISDC_REACTION_ALLEN_CAHN)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "unknown reaction %d", o.reaction);
  if (o.max_sweeps < 1 || o.max_sweeps > 100000 || o.mg_max_cycles < 1)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "max_sweeps and mg_max_cycles must be >= 1");
  if (o.temporal_blocking < -1 || o.temporal_blocking > 2)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "temporal_blocking must be -1, 0, 1 or 2");
  {
    const int r = o.rb_run;
    const bool ok = r == 0 || r == -1 || r == -2 || r == -4 || r == -8 || r == 1 || r == 2 || r == 4 || r == 8 ||
                    r == 16 || r == 32;
    if (!ok) return fail(nullptr, ISDC_ERR_INVALID_ARG, "rb_run must be 0, 1, 2, 4, 8, 16, 32, -1, -2, -4 or -8");
  }
  if (o.use_graphs < 0 || o.use_graphs > 2) return fail(nullptr, ISDC_ERR_INVALID_ARG, "use_graphs must be 0, 1 or 2");
  if (o.fused_transfer < -1 || o.fused_transfer > 1)
    return fail(nullptr, ISDC_ERR_INVALID_ARG, "fused_transfer must be -1, 0 or 1");
  if (o.stencil != 0 && o.stencil != 1) return fail(nullptr, ISDC_ERR_INVALID_ARG, "unknown stencil %d", o.stencil);
  if (o.stencil == 1 && (ndim != 2 || o.smoother != ISDC_SMOOTHER_JACOBI || o.vcycle_fp32 || o.equation != 0))
    return fail(nullptr, ISDC_ERR_UNSUPPORTED,
                "the compact stencil is implemented in 2D with damped-Jacobi smoothing and FP64 V-cycles");
  if (o.equation == 1 && o.vcycle_fp32)
    return fail(nullptr, ISDC_ERR_UNSUPPORTED, "viscous Burgers is implemented with FP64 V-cycles");

  isdc_ctx* ctx = new isdc_ctx();
  ctx->dim = ndim;
  ctx->n = int(n);
  ctx->N = pow_dim(ndim, size_t(n));
  ctx->M = M;
  ctx->node_kind = int(nodes);
  ctx->off = nodes == ISDC_NODES_GAUSS_LOBATTO ? 0 : 1;
  ctx->P = M + ctx->off;
  ctx->nu = nu;
  ctx->dt = dt;
  ctx->equation = o.equation;
  ctx->h = o.equation == 1 ? 2.0 / double(n) : 1.0 / double(n + 1);
  ctx->opt = o;
  ctx->stencil = o.stencil;
  auto bail = [&](isdc_status st) {
    snprintf(g_create_error, sizeof g_create_error, "%s", ctx->err);
    isdc_destroy(ctx);
    return st;
  };
  if (o.stream) {
    ctx->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      fail(ctx, ISDC_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
      return bail(ISDC_ERR_CUDA);
    }
    ctx->own_stream = true;
  }
  isdc_collocation_tables(nodes, M, ctx->tau, ctx->Q, ctx->S);
  const int P = ctx->P, off = ctx->off;
  double tpt[kMaxP];  // t_p - T_n over dt: 0, then the nodes
  tpt[0] = 0.0;
  for (int m = 0; m < M; ++m) tpt[m + off] = ctx->tau[m];
  ctx->tables.M = M;
  ctx->tables.P = P;
  for (int p = 0; p < P; ++p)
    for (int j = 0; j < M; ++j) ctx->tables.dtQ[p][j] = p - off >= 0 ? dt * ctx->Q[(p - off) * M + j] : 0.0;
  for (int m = 0; m < P - 1; ++m) ctx->tables.dtm[m] = dt * (tpt[m + 1] - tpt[m]);
  double w[kMaxM];
  end_weights(M, ctx->tau, w);
  ctx->ends.M = M;
  for (int j = 0; j < M; ++j) ctx->ends.dtw[j] = dt * w[j];

  const size_t N = ctx->N;
  isdc_status st;
#define CREATE_TRY(call)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) {                                  \
      isdc_status s_ = e_ == cudaErrorMemoryAllocation ? ISDC_ERR_OOM : ISDC_ERR_CUDA; \
      fail(ctx, s_, "%s: %s", #call, cudaGetErrorString(e_)); \
      return bail(s_);                                        \
    }                                                         \
  } while (0)
  CREATE_TRY(cudaMalloc(&ctx->U, size_t(P) * N * sizeof(double)));
  CREATE_TRY(cudaMalloc(&ctx->F, size_t(P) * N * sizeof(double)));
  CREATE_TRY(cudaMalloc(&ctx->C, size_t(P - 1) * N * sizeof(double)));
  if (ctx->stencil != 1) CREATE_TRY(cudaMalloc(&ctx->FE, size_t(P) * N * sizeof(double)));
  if (ctx->stencil == 1) {
    CREATE_TRY(cudaMalloc(&ctx->G, size_t(P) * N * sizeof(double)));
    CREATE_TRY(cudaMalloc(&ctx->Rs, 3 * size_t(P - 1) * N * sizeof(double)));
  }
  CREATE_TRY(cudaMalloc(&ctx->b, N * sizeof(double)));
  CREATE_TRY(cudaMalloc(&ctx->d_scal, 4 * sizeof(unsigned long long)));
  CREATE_TRY(cudaMemset(ctx->d_scal, 0, 4 * sizeof(unsigned long long)));
  CREATE_TRY(cudaMallocHost(&ctx->h_scal, 4 * sizeof(unsigned long long)));
  ctx->hist_cap = std::max(o.max_sweeps, 1) + 1;
  CREATE_TRY(cudaMallocHost(&ctx->h_hist, size_t(ctx->hist_cap) * sizeof(unsigned long long)));
  if (o.vcycle_fp32) {
    if ((st = alloc_hier(ctx, ctx->h32, true)) != ISDC_OK) return bail(st);
    if (o.smoother == ISDC_SMOOTHER_RBGS && o.nu1 >= 1 && o.nu2 >= 1 && ctx->h32.lb > 0) {
      ctx->hn = size_t((n + 1) / 2) * (ndim == 2 ? size_t(n) : size_t(n) * size_t(n));
      CREATE_TRY(cudaMalloc(&ctx->sp_x, 2 * ctx->hn * sizeof(float)));
      CREATE_TRY(cudaMalloc(&ctx->sp_b, 2 * ctx->hn * sizeof(float)));
      CREATE_TRY(cudaMalloc(&ctx->sp_r, ctx->hn * sizeof(float)));
      // padding slots (past the last point of a row) are never written: keep them zero
      CREATE_TRY(cudaMemset(ctx->sp_x, 0, 2 * ctx->hn * sizeof(float)));
      CREATE_TRY(cudaMemset(ctx->sp_b, 0, 2 * ctx->hn * sizeof(float)));
      CREATE_TRY(cudaMemset(ctx->sp_r, 0, ctx->hn * sizeof(float)));
      if (ndim == 3) {
        CREATE_TRY(cudaMalloc(&ctx->sp_xb, ctx->hn * sizeof(float)));
        CREATE_TRY(cudaMemset(ctx->sp_xb, 0, ctx->hn * sizeof(float)));
        // the blocked passes stage their planes in more than the default 48 KB
        CREATE_TRY(cudaFuncSetAttribute(k_rbgs_split_tb<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(TbShape<2>::smem_bytes)));
        CREATE_TRY(cudaFuncSetAttribute(k_rbgs_split_tb<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(TbShape<4>::smem_bytes)));
      }
    }
    if (ndim == 2) configure_bottom<float, 2>(ctx->h32); else configure_bottom<float, 3>(ctx->h32);
    for (int m = 0; m < P - 1; ++m)
      if ((st = upload_ainv(ctx, ctx->h32, m, ctx->tables.dtm[m] * nu)) != ISDC_OK) return bail(st);
  } else {
    if ((st = alloc_hier(ctx, ctx->h64, false)) != ISDC_OK) return bail(st);
    if (ctx->stencil == 1) {
      cudaFuncSetAttribute(k_bottom9, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctx->h64.bottom_smem));
    } else if (ctx->equation == 1) {
      if (ndim == 2)
        cudaFuncSetAttribute(k_bottom_per<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctx->h64.bottom_smem));
      else
        cudaFuncSetAttribute(k_bottom_per<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctx->h64.bottom_smem));
    } else {
      if (ndim == 2) configure_bottom<double, 2>(ctx->h64); else configure_bottom<double, 3>(ctx->h64);
    }
    for (int m = 0; m < P - 1; ++m)
      if ((st = upload_ainv(ctx, ctx->h64, m, ctx->tables.dtm[m] * nu)) != ISDC_OK) return bail(st);
  }
  ctx->spare_slot = P - 1;
  if ((st = tune_smoother(ctx)) != ISDC_OK) return bail(st);
  if ((st = setup_transfer(ctx)) != ISDC_OK) return bail(st);
  CREATE_TRY(cudaGetLastError());
#undef CREATE_TRY
  *out = ctx;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_step(isdc_ctx* ctx, double* u, int n_sweeps, int n_vcycles) {
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  if (!u) return fail(ctx, ISDC_ERR_INVALID_ARG, "u is NULL");
  if (n_sweeps < 0 || n_vcycles < 0) return fail(ctx, ISDC_ERR_INVALID_ARG, "n_sweeps and n_vcycles must be >= 0");
  return ctx->dim == 2 ? run_step<2>(ctx, u, n_sweeps, n_vcycles) : run_step<3>(ctx, u, n_sweeps, n_vcycles);
}

ISDC_API isdc_status isdc_step_host(isdc_ctx* ctx, double* u_host, int n_sweeps, int n_vcycles) {
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  if (!u_host) return fail(ctx, ISDC_ERR_INVALID_ARG, "u_host is NULL");
  if (!ctx->u_dev) CUDA_TRY(ctx, cudaMalloc(&ctx->u_dev, ctx->N * sizeof(double)));
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->u_dev, u_host, ctx->N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  isdc_status st = isdc_step(ctx, ctx->u_dev, n_sweeps, n_vcycles);
  if (st != ISDC_OK && st != ISDC_ERR_NOT_CONVERGED && st != ISDC_ERR_NONFINITE) return st;
  CUDA_TRY(ctx, cudaMemcpyAsync(u_host, ctx->u_dev, ctx->N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return st;
}

ISDC_API isdc_status isdc_residual(const isdc_ctx* cctx, double* res) {
  isdc_ctx* ctx = const_cast<isdc_ctx*>(cctx);
  if (!ctx || !res) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  *res = bits_to_double(ctx->h_scal[0]);
  return ISDC_OK;
}

ISDC_API isdc_status isdc_stats(const isdc_ctx* cctx, int* sweeps, int64_t* vcycles) {
  isdc_ctx* ctx = const_cast<isdc_ctx*>(cctx);
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (sweeps) *sweeps = ctx->last_sweeps;
  if (vcycles) *vcycles = ctx->last_vcycles;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_residual_history(const isdc_ctx* cctx, double* hist, int cap, int* count) {
  isdc_ctx* ctx = const_cast<isdc_ctx*>(cctx);
  if (!ctx || (!hist && cap > 0)) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const int c = std::min(cap, ctx->hist_count);
  for (int q = 0; q < c; ++q) hist[q] = bits_to_double(ctx->h_hist[q]);
  if (count) *count = ctx->hist_count;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_set_record_history(isdc_ctx* ctx, int record) {
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  ctx->record_history = record ? 1 : 0;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_get_nodes(const isdc_ctx* cctx, double* dst) {
  isdc_ctx* ctx = const_cast<isdc_ctx*>(cctx);
  if (!ctx || !dst) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaMemcpyAsync(dst, ctx->U + size_t(ctx->off) * ctx->N, size_t(ctx->M) * ctx->N * sizeof(double),
                                cudaMemcpyDeviceToDevice, ctx->stream));
  return ISDC_OK;
}

ISDC_API isdc_status isdc_set_nodes(isdc_ctx* ctx, const double* src) {
  if (!ctx || !src) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->U + size_t(ctx->off) * ctx->N, src, size_t(ctx->M) * ctx->N * sizeof(double),
                                cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->nodes_pending = 1;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_vcycles(isdc_ctx* ctx, double a, double* x, const double* b, int n_cycles) {
  if (!ctx || !x || !b) return ISDC_ERR_INVALID_ARG;
  if (!(a > 0) || !std::isfinite(a) || n_cycles < 0) return fail(ctx, ISDC_ERR_INVALID_ARG, "need a > 0, n_cycles >= 0");
  isdc_status st;
  if (ctx->opt.vcycle_fp32) st = upload_ainv(ctx, ctx->h32, ctx->spare_slot, a);
  else st = upload_ainv(ctx, ctx->h64, ctx->spare_slot, a);
  if (st != ISDC_OK) return st;
  if (ctx->equation == 1) {  // periodic (I - a L_h) x = b, row-scaled by d
    k_scale<double><<<4 * 152, 256, 0, ctx->stream>>>(ctx->N, 1.0 / coef_per(ctx->dim, ctx->n, a).d, b, ctx->b);
    LAUNCH_CHECK(ctx);
    for (int c = 0; c < n_cycles; ++c)
      if ((st = ctx->dim == 2 ? vcycle_per<2>(ctx, ctx->spare_slot, a, x, ctx->b)
                              : vcycle_per<3>(ctx, ctx->spare_slot, a, x, ctx->b)) != ISDC_OK)
        return st;
    return ISDC_OK;
  }
  if (ctx->stencil == 1) {  // (W - a L_9) x = b, row-scaled by c0
    k_scale<double><<<4 * 152, 256, 0, ctx->stream>>>(ctx->N, 1.0 / coef9(ctx->n, a).c0, b, ctx->b);
    LAUNCH_CHECK(ctx);
    for (int c = 0; c < n_cycles; ++c)
      if ((st = vcycle9(ctx, ctx->spare_slot, a, x, ctx->b)) != ISDC_OK) return st;
    return ISDC_OK;
  }
  // the V-cycles act on the row-scaled system: beta = b / d (in the context's rhs buffer)
  const double d0 = level_coef(ctx->dim, ctx->n, a).d;
  k_scale<double><<<4 * 152, 256, 0, ctx->stream>>>(ctx->N, 1.0 / d0, b, ctx->b);
  LAUNCH_CHECK(ctx);
  return ctx->dim == 2 ? node_solve<2>(ctx, ctx->spare_slot, a, x, ctx->b, n_cycles)
                       : node_solve<3>(ctx, ctx->spare_slot, a, x, ctx->b, n_cycles);
}

ISDC_API isdc_status isdc_profile_enable(isdc_ctx* ctx, int enable) {
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  prof_flush(ctx);
  Profiler& P = ctx->prof;
  if (enable) {
    std::fill(P.ms, P.ms + PC_COUNT, 0.0);
    std::fill(P.bytes, P.bytes + PC_COUNT, 0.0);
    std::fill(P.dp_ops, P.dp_ops + PC_COUNT, 0.0);
    std::fill(P.sp_ops, P.sp_ops + PC_COUNT, 0.0);
    std::fill(P.launches, P.launches + PC_COUNT, 0LL);
  }
  P.on = enable != 0;
  P.event_mask = unsigned(enable) & ((1u << PC_COUNT) - 1u);
  return ISDC_OK;
}

ISDC_API isdc_status isdc_profile_read(isdc_ctx* ctx, isdc_kernel_stat* out, int cap, int* count) {
  if (!ctx || (!out && cap > 0)) return ISDC_ERR_INVALID_ARG;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  const Profiler& P = ctx->prof;
  int c = 0;
  for (int k = 0; k < PC_COUNT; ++k) {
    if (!P.launches[k]) continue;
    if (c < cap) {
      isdc_kernel_stat& o = out[c];
      std::memset(&o, 0, sizeof o);
      snprintf(o.name, sizeof o.name, "%s", kProfNames[k]);
      o.launches = P.launches[k];
      o.total_ms = (P.event_mask & (1u << k)) ? P.ms[k] : -1.0;
      o.bytes = P.bytes[k];
      o.fp64_ops = P.dp_ops[k];
      o.fp32_ops = P.sp_ops[k];
    }
    ++c;
  }
  if (count) *count = c;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_tuning(const isdc_ctx* ctx, int* zb_fp64, int* zb_fp32, int* tb_depth, int* tb_planes) {
  if (!ctx) return ISDC_ERR_INVALID_ARG;
  if (zb_fp64) *zb_fp64 = ctx->zb64;
  if (zb_fp32) *zb_fp32 = ctx->zb32;
  if (tb_depth) *tb_depth = ctx->tb_depth;
  if (tb_planes) *tb_planes = ctx->tb_zc;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_tuning_transfer(const isdc_ctx* ctx, int* kc, int max_levels, int* n_levels) {
  if (!ctx || (!kc && max_levels > 0) || max_levels < 0) return ISDC_ERR_INVALID_ARG;
  const bool fp32 = ctx->opt.vcycle_fp32 != 0;
  const int lb = ctx->stencil == 1 || ctx->equation == 1 ? 0 : (fp32 ? ctx->h32.lb : ctx->h64.lb);
  for (int l = 0; l < lb && l < max_levels; ++l)
    kc[l] = (l == 0 && ctx->sp_x) ? ctx->rr_split : (fp32 ? ctx->rr32 : ctx->rr64)[l];
  if (n_levels) *n_levels = lb;
  return ISDC_OK;
}

ISDC_API const char* isdc_last_error(const isdc_ctx* ctx) { return ctx ? ctx->err : g_create_error; }
