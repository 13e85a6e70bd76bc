// batch.cu -- the batched / continuously batched ISDC engine (isdc_batch_*).
//
// An engine holds up to kMaxInst independent ISDC integrations of one spatial
// dimension, each with its own side n, nu, M, dt and number of time steps.
// A tick advances every running instance by one SDC sweep (Sec. 2, Eq. 4;
// Sec. 3): instances that start a time step are spread first, then the node
// solves run with L FP32 V-cycles in defect-correction form (FP64 node state,
// quadrature term, node residual and SDC residual), then every instance's SDC
// residual is read back.  Each phase of the tick is one persistent
// grid-stride launch over the work list of all instances taking part, and the
// whole tick is one CUDA graph, captured once: the work lists live in device
// memory and are rewritten before each launch, so instances can be admitted
// and retired between ticks without re-capture (continuous batching).  Device
// memory for an instance is taken with cudaMallocAsync when it is admitted,
// within an HBM budget, and returned when its result is taken.
//
// Autotuning: the first ticks run with different launch shapes (threads per
// block = tile size, persistent blocks per SM, one cooperative launch), then
// with 2..4 lanes of the fastest graph shape, each lane's launches taking all
// or 1/lanes of its blocks per SM, the latter also with staggered lanes; each
// tick's DOF-sweep rate is measured with events and the fastest shape is kept
// for the engine's life.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/isdc.h"
#include "batch_kernels.cuh"
#include "host_util.h"

#define ISDC_API extern "C" __attribute__((visibility("default")))

using namespace isdc;
using namespace isdc::batch;

namespace {

thread_local char g_batch_error[512] = "";

// Work-list kinds per (node solve, level): every point, coarse points and
// coarse cells (one thread each); fused 2D tiles; rows of the level, of its
// coarse grid and of its coarse cells (one warp each).
enum ListKind {
  LK_FULL = 0, LK_CPTS = 1, LK_CELLS = 2, LK_TILE = 3, LK_ROWS = 4, LK_CROWS = 5, LK_CELLROWS = 6, LK_KINDS = 7
};

struct Slot {
  int state = ISDC_SLOT_FREE;
  int n = 0, M = 0, nlev = 0, steps = 0, steps_done = 0, sweeps = 0, total_sweeps = 0, nonconverged = 0;
  bool spread_next = false;
  double last_res = 0.0;
  size_t bytes = 0;
  void* mem = nullptr;
};

// Launch shape of the grid-wide phases: threads per block (the point-wise
// phases' tile; the fused 2D phases' tile is 32 x threads/32 coarse points;
// the row-structured phases' tile is threads/32 rows), blocks per SM, whether
// the whole tick is one persistent cooperative launch (fused 2D mode only;
// blocks per SM from the occupancy calculator) instead of a graph of one
// launch per phase, and the number of lanes: the running instances are dealt
// to that many independent chains of the tick graph (balanced by work), which
// the graph runs concurrently, so one lane's FP64-bound phases overlap another
// lane's HBM-bound V-cycle phases.  Every shape gives the same result bit for
// bit, so the autotuner's trial ticks are real sweeps.
// With split set, each lane's launches take blocks_per_sm / lanes blocks per
// SM (rounded up), so the lanes' blocks are resident side by side and an
// FP64-bound phase of one lane shares the SMs with an HBM-bound phase of
// another; without it every launch takes the whole blocks_per_sm.  With
// stagger set, lane q starts once lane q-1's first right-hand-side phase has
// completed, so the lanes run a phase apart instead of in step.
struct Shape {
  int threads, blocks_per_sm, persistent, lanes, split, stagger;
};
constexpr int kMaxLanes = 4;
// the autotuner's first candidates (one lane); lane counts 2..kMaxLanes of the
// fastest graph shape, whole, split, and split and staggered, are appended
// once these have run
const Shape kBaseShapes[] = {{256, 8, 0, 1, 0, 0}, {128, 16, 0, 1, 0, 0}, {512, 4, 0, 1, 0, 0},
                             {256, 16, 0, 1, 0, 0}, {128, 8, 0, 1, 0, 0}, {256, 0, 1, 1, 0, 0},
                             {512, 0, 1, 1, 0, 0}};
constexpr int kNumBase = int(sizeof(kBaseShapes) / sizeof(kBaseShapes[0]));
constexpr int kMaxCands = kNumBase + 3 * (kMaxLanes - 1);

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

struct isdc_batch {
  int dim = 0, L = 2, Mmax = 0, Lmax = 0, sms = 0, max_side = 0;
  int fused = 0;  // 2D damped Jacobi: smoother fused into the transfer passes (temporal-blocking depth 1)
  isdc_options opt{};
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Inst* d_insts = nullptr;
  Inst* h_insts = nullptr;  // pinned mirror
  List* d_lists = nullptr;
  List* h_lists = nullptr;  // pinned staging
  int nlists = 0;
  unsigned long long *d_rbits = nullptr, *d_dummy = nullptr, *h_rbits = nullptr;
  Slot slots[kMaxInst];
  // autotuner candidates, with a graph per graph shape
  Shape cands[kMaxCands] = {};
  int ncands = 0;
  bool lanes_added = false;  // lane-count candidates appended
  cudaGraphExec_t exec[kMaxCands] = {};
  int shape = 0;         // candidate in use
  int tuned = 0;         // 1 once the autotuner has chosen
  int tune_next = 0;     // next candidate to try
  bool tune_warm = false;  // the first tick (every instance's spread) is run but not scored
  double tune_rate[kMaxCands] = {};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // lanes 1.. of a multi-lane tick graph: their capture streams, fork and join events
  cudaStream_t lane_st[kMaxLanes - 1] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxLanes - 1] = {};
  cudaEvent_t ev_stage[kMaxLanes - 1] = {};  // lane q's first right-hand side done (staggered lanes)
  long long ticks = 0;
  long long kernel_launches = 0;   // kernel nodes executed by all ticks
  double last_tick_bytes = 0.0;    // algorithmic bytes of the last tick (tick_bytes)
  int kernel_nodes[kMaxCands] = {};  // kernel nodes per tick graph
  // persistent tick: phase table, grid barrier, resident blocks per SM per shape
  Phase* d_phases = nullptr;
  int nphases = 0;
  GridBarrier *d_gb = nullptr, *h_gb = nullptr;
  int pers_bps[kMaxCands] = {};
  char err[512] = "";
};

namespace {

isdc_status bfail(isdc_batch* b, isdc_status st, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define B_TRY(b, call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? ISDC_ERR_OOM : ISDC_ERR_CUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                         \
  } while (0)

int levels_of(int n) {
  int l = 1;
  while (n > 3) { n = (n - 1) / 2; ++l; }
  return l;
}

size_t pts(int dim, int n) { return dim == 2 ? size_t(n) * n : size_t(n) * n * n; }

int list_index(const isdc_batch* b, int m, int l, int kind) { return ((m * b->Lmax) + l) * LK_KINDS + kind; }
int list_coarse(const isdc_batch* b, int m) { return (b->Mmax - 1) * b->Lmax * LK_KINDS + m; }
int list_bottom(const isdc_batch* b, int m) { return (b->Mmax - 1) * b->Lmax * LK_KINDS + (b->Mmax - 1) + m; }
int list_spread(const isdc_batch* b) { return (b->Mmax - 1) * b->Lmax * LK_KINDS + 2 * (b->Mmax - 1); }
// instances with M nodes (2 <= M <= Mmax): those starting a step, all running ones
int list_spread_m(const isdc_batch* b, int M) { return list_spread(b) + 1 + (M - 2); }
int list_sweep_m(const isdc_batch* b, int M) { return list_spread(b) + 1 + (b->Mmax - 1) + (M - 2); }
int bottom_side(int dim) { return dim == 2 ? kBatchBottom2 : kBatchBottom3; }
int bottom_level(int dim, int n) {  // first level of side <= the bottom threshold
  int l = 0;
  while (n > bottom_side(dim)) { n = (n - 1) / 2; ++l; }
  return l;
}
size_t bottom_smem(int dim) {  // 3 FP32 arrays per level from the threshold side down to 3
  size_t s = 0;
  for (int n = bottom_side(dim); n >= 3; n = (n - 1) / 2) s += 3 * pts(dim, n) * 4;
  return s;
}

// Bytes of device memory one instance needs (node state FP64, hierarchy FP32).
size_t instance_bytes(const isdc_batch* b, int n, int M) {
  const size_t N = pts(b->dim, n);
  size_t s = 0;
  s += align256(size_t(M) * N * 8);        // U
  s += align256(size_t(M) * N * 8);        // F
  s += align256(size_t(M - 1) * N * 8);    // C
  const int nlev = levels_of(n);
  int side = n;
  const int per_level = b->opt.smoother == ISDC_SMOOTHER_JACOBI ? 4 : 3;
  for (int l = 0; l < nlev; ++l) {
    s += per_level * align256(pts(b->dim, side) * 4);
    side = (side - 1) / 2;
  }
  s += align256(size_t(M - 1) * (b->dim == 2 ? 81 : 729) * 4);  // coarse inverses
  return s;
}

enum TickMode { MODE_LEGACY = 0, MODE_FUSED2D = 1, MODE_RB_BOTTOM = 2 };

// How a tick runs its V-cycles.  Fused 2D damped Jacobi (V(1, nu2 <= 1)):
// one fused pass per leg and grid-wide level, the coarse levels in one block
// per instance.  Red-black Gauss-Seidel: the separate phases on the grid-wide
// levels as row-structured passes, the coarse levels in one block per
// instance.  Otherwise (damped Jacobi outside the fused form): every phase of
// every level as its own point-wise pass.
int tick_mode(const isdc_batch* b, const Shape&) {
  const bool jac = b->opt.smoother == ISDC_SMOOTHER_JACOBI;
  if (!jac) return MODE_RB_BOTTOM;
  return b->fused ? MODE_FUSED2D : MODE_LEGACY;
}

// Rebuild every work list for the current running set and launch shape.  With
// several lanes, lane q's lists start at h_lists + q * nlists, and each running
// instance goes to the lane with the least work so far (largest instances
// first; work ~ points x node solves, M - 1).
void build_lists(isdc_batch* b, const Shape& sh) {
  const int tile = sh.threads, ty = sh.threads / 32;
  const int mode = tick_mode(b, sh);
  for (int q = 0; q < b->nlists * sh.lanes; ++q) {
    b->h_lists[q].count = 0;
    b->h_lists[q].total = 0;
    b->h_lists[q].start[0] = 0;
  }
  int lane_of[kMaxInst];
  {
    int order[kMaxInst], cnt = 0;
    for (int i = 0; i < kMaxInst; ++i)
      if (b->slots[i].state == ISDC_SLOT_RUNNING) order[cnt++] = i;
    auto work = [&](int i) { return double(pts(b->dim, b->slots[i].n)) * (b->slots[i].M - 1); };
    std::stable_sort(order, order + cnt, [&](int x, int y) { return work(x) > work(y); });
    double load[kMaxLanes] = {};
    for (int c = 0; c < cnt; ++c) {
      int best = 0;
      for (int q = 1; q < sh.lanes; ++q)
        if (load[q] < load[best]) best = q;
      lane_of[order[c]] = best;
      load[best] += work(order[c]);
    }
  }
  int lane = 0;  // lane of the instance being added
  auto add_tiles = [&](int li, int inst, int tiles) {
    List& L = b->h_lists[lane * b->nlists + li];
    L.inst[L.count] = inst;
    L.start[L.count] = L.total;
    L.total += tiles;
    L.count += 1;
    L.start[L.count] = L.total;
  };
  auto add = [&](int li, int inst, size_t domain) { add_tiles(li, inst, int((domain + tile - 1) / tile)); };
  const int dim = b->dim;
  for (int i = 0; i < kMaxInst; ++i) {
    const Slot& S = b->slots[i];
    if (S.state != ISDC_SLOT_RUNNING) continue;
    lane = lane_of[i];
    const size_t N = pts(dim, S.n);
    if (S.spread_next) {
      add(list_spread(b), i, N);
      add(list_spread_m(b, S.M), i, N);
    }
    add(list_sweep_m(b, S.M), i, N);
    // grid-wide levels: every level above the coarsest (separate phases) or
    // the levels above the per-instance bottom block
    const int grid_levels = mode == MODE_LEGACY ? S.nlev - 1 : bottom_level(dim, S.n);
    for (int m = 0; m < S.M - 1; ++m) {
      add(list_coarse(b, m), i, dim == 2 ? 9 : 27);
      add_tiles(list_bottom(b, m), i, 1);
      int side = S.n;
      auto add_rows = [&](int li, int s) { add_tiles(li, i, int(((dim == 2 ? s : s * s) + ty - 1) / ty)); };
      for (int l = 0; l < S.nlev - 1; ++l) {
        const int sc = (side - 1) / 2;
        if (l == 0 || (mode == MODE_LEGACY && l < grid_levels))  // level 0: rhs, update
          add(list_index(b, m, l, LK_FULL), i, pts(dim, side));
        if (l < grid_levels) {
          if (mode == MODE_LEGACY) {
            add(list_index(b, m, l, LK_CPTS), i, pts(dim, sc));
            add(list_index(b, m, l, LK_CELLS), i, pts(dim, sc + 1));
          } else if (mode == MODE_FUSED2D) {
            add_tiles(list_index(b, m, l, LK_TILE), i, ((sc + kFtX - 1) / kFtX) * ((sc + ty - 1) / ty));
          } else {
            add_rows(list_index(b, m, l, LK_ROWS), side);
            add_rows(list_index(b, m, l, LK_CROWS), sc);
            add_rows(list_index(b, m, l, LK_CELLROWS), sc + 1);
          }
        }
        side = sc;
      }
    }
  }
}

// Algorithmic bytes of one tick for the running set (each phase reads each
// input stream once and writes each output once; FP64 node state, FP32
// levels).  Used for the engine's roofline.
double tick_bytes(const isdc_batch* b, const Shape& sh) {
  const int mode = tick_mode(b, sh), dim = b->dim;
  const bool jac = b->opt.smoother == ISDC_SMOOTHER_JACOBI;
  const int nu1 = b->opt.nu1, nu2 = b->opt.nu2;
  double total = 0.0;
  for (int i = 0; i < kMaxInst; ++i) {
    const Slot& S = b->slots[i];
    if (S.state != ISDC_SLOT_RUNNING) continue;
    const double N = double(pts(dim, S.n));
    const int M = S.M;
    double t = (3.0 * M - 1.0) * 8.0 * N;                 // sweep end
    if (S.spread_next) t += 2.0 * M * 8.0 * N;            // spread
    const int grid_levels = mode == MODE_LEGACY ? S.nlev - 1 : bottom_level(dim, S.n);
    double cyc = 0.0;                                     // one V-cycle, FP32
    int side = S.n;
    for (int l = 0; l < grid_levels; ++l) {
      const double Nl = double(pts(dim, side)), Nc = double(pts(dim, (side - 1) / 2));
      if (mode == MODE_FUSED2D) {
        cyc += 4.0 * (3.0 * Nl + Nc) + (l > 0 ? 0.0 : 4.0 * Nl);  // down: x (not from zero), b, t; b_c
        cyc += 4.0 * ((nu2 ? 3.0 : 2.0) * Nl + Nc);                // up: t, b, x; e_c
      } else if (!jac) {
        cyc += 4.0 * ((nu1 + nu2) * 2.0 * 1.5 * Nl + 2.0 * Nl + (0.5 * Nl + Nc) + (Nl + Nc));
      } else {
        cyc += 4.0 * ((nu1 + nu2) * 3.0 * Nl + 3.0 * Nl + (Nl + Nc) + (Nl + Nc));
      }
      side = (side - 1) / 2;
    }
    if (mode != MODE_LEGACY) cyc += 4.0 * 3.0 * double(pts(dim, side));  // bottom block: b, x in, x out
    t += (M - 1) * (28.0 * N + 20.0 * N + b->L * cyc);                    // rhs, update, L cycles per node
    total += t;
  }
  return total;
}

template <int DIM>
void launch_sweep_end(int M, dim3 grid, dim3 blk, cudaStream_t st, const Inst* I, const List* L, int reaction,
                      unsigned long long* rbits) {
  switch (M) {
    case 2: kb_sweep_end<DIM, 2><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
    case 3: kb_sweep_end<DIM, 3><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
    case 4: kb_sweep_end<DIM, 4><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
    case 5: kb_sweep_end<DIM, 5><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
    case 6: kb_sweep_end<DIM, 6><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
    default: kb_sweep_end<DIM, 7><<<grid, blk, 0, st>>>(I, L, reaction, rbits); break;
  }
}

// Record one lane's launches of a tick on stream st, over the lane's work
// lists Ls (inside a capture).
template <int DIM>
void record_lane(isdc_batch* b, const Shape& sh, cudaStream_t st, const List* Ls, cudaEvent_t after_rhs0) {
  const int bps = sh.split ? (sh.blocks_per_sm + sh.lanes - 1) / sh.lanes : sh.blocks_per_sm;
  const dim3 grid(bps * b->sms), blk(sh.threads);
  const Inst* I = b->d_insts;
  const int reaction = b->opt.reaction;
  const bool jac = b->opt.smoother == ISDC_SMOOTHER_JACOBI;
  const int nu1 = b->opt.nu1, nu2 = b->opt.nu2;
  const float omega = float(b->opt.omega);
  const int mode = tick_mode(b, sh);
  const int ty = sh.threads / 32;
  const int par = (nu1 + nu2) & 1;  // Jacobi: a level's iterate ends in t after an odd sweep count
  kb_spread<DIM><<<grid, blk, 0, st>>>(I, Ls + list_spread(b), reaction);
  for (int M = 2; M <= b->Mmax; ++M)
    launch_sweep_end<DIM>(M, grid, blk, st, I, Ls + list_spread_m(b, M), reaction, b->d_dummy);
  for (int m = 0; m < b->Mmax - 1; ++m) {
    const List* full0 = Ls + list_index(b, m, 0, LK_FULL);
    kb_rhs<DIM><<<grid, blk, 0, st>>>(I, full0, m, reaction);
    if (m == 0 && after_rhs0) cudaEventRecord(after_rhs0, st);
    int loc0 = 0;  // level-0 error: in x (0) or t (1)
    if (mode != MODE_LEGACY) {
      const int Lg = bottom_level(DIM, b->max_side);
      for (int c = 0; c < b->L; ++c) {
        for (int l = 0; l < Lg; ++l) {
          const int zero = (l > 0 || c == 0) ? 1 : 0;
          if (mode == MODE_FUSED2D) {
            const List* tl = Ls + list_index(b, m, l, LK_TILE);
            if (ty == 4) kb_down2<4><<<grid, 128, 0, st>>>(I, tl, m, l, omega, zero);
            else if (ty == 8) kb_down2<8><<<grid, 256, 0, st>>>(I, tl, m, l, omega, zero);
            else kb_down2<16><<<grid, 512, 0, st>>>(I, tl, m, l, omega, zero);
          } else {
            const List* rows = Ls + list_index(b, m, l, LK_ROWS);
            for (int s = 0; s < nu1; ++s) {
              kb_rbgs_rows<DIM><<<grid, blk, 0, st>>>(I, rows, m, l, 0, zero && s == 0);
              kb_rbgs_rows<DIM><<<grid, blk, 0, st>>>(I, rows, m, l, 1, 0);
            }
            kb_residual_red_rows<DIM><<<grid, blk, 0, st>>>(I, rows, m, l);
            kb_restrict_red_rows<DIM><<<grid, blk, 0, st>>>(I, Ls + list_index(b, m, l, LK_CROWS), m, l);
          }
        }
        kb_bottom<DIM><<<kMaxInst, kBottomThreads, bottom_smem(DIM), st>>>(I, Ls + list_bottom(b, m), m, c > 0 ? 1 : 0,
                                                                          jac ? 0 : 1, nu1, nu2, omega);
        for (int l = Lg - 1; l >= 0; --l) {
          if (mode == MODE_FUSED2D) {
            const List* tl = Ls + list_index(b, m, l, LK_TILE);
            if (ty == 4) kb_up2<4><<<grid, 128, 0, st>>>(I, tl, m, l, omega, nu2);
            else if (ty == 8) kb_up2<8><<<grid, 256, 0, st>>>(I, tl, m, l, omega, nu2);
            else kb_up2<16><<<grid, 512, 0, st>>>(I, tl, m, l, omega, nu2);
          } else {
            const List* rows = Ls + list_index(b, m, l, LK_ROWS);
            const List* cells = Ls + list_index(b, m, l, LK_CELLROWS);
            if (nu2 >= 1) kb_prolong_rows<DIM, true><<<grid, blk, 0, st>>>(I, cells, l);
            else kb_prolong_rows<DIM, false><<<grid, blk, 0, st>>>(I, cells, l);
            for (int s = 0; s < nu2; ++s) {
              kb_rbgs_rows<DIM><<<grid, blk, 0, st>>>(I, rows, m, l, 0, 0);
              kb_rbgs_rows<DIM><<<grid, blk, 0, st>>>(I, rows, m, l, 1, 0);
            }
          }
        }
      }
    } else {  // damped Jacobi, every phase of every level as its own pass
      for (int c = 0; c < b->L; ++c) {
        for (int l = 0; l < b->Lmax - 1; ++l) {
          const bool zero = l > 0 || c == 0;
          const List* full = Ls + list_index(b, m, l, LK_FULL);
          int loc = l == 0 ? loc0 : 0;
          for (int s = 0; s < nu1; ++s) {
            kb_jacobi<DIM><<<grid, blk, 0, st>>>(I, full, m, l, omega, loc, zero && s == 0);
            loc ^= 1;
          }
          kb_residual<DIM><<<grid, blk, 0, st>>>(I, full, m, l, loc);
          kb_restrict<DIM, false><<<grid, blk, 0, st>>>(I, Ls + list_index(b, m, l, LK_CPTS), m, l);
        }
        // every instance's coarsest grid; the result goes where a smoothed level's
        // iterate would be (t after an odd sweep count) so the prolongation reads
        // one location for all instances
        kb_coarse<DIM><<<grid, blk, 0, st>>>(I, Ls + list_coarse(b, m), m, par);
        for (int l = b->Lmax - 2; l >= 0; --l) {
          int loc = (l == 0 ? loc0 : 0) ^ (nu1 & 1);
          kb_prolong<DIM, false><<<grid, blk, 0, st>>>(I, Ls + list_index(b, m, l, LK_CELLS), l, loc, par);
          for (int s = 0; s < nu2; ++s) {
            kb_jacobi<DIM><<<grid, blk, 0, st>>>(I, Ls + list_index(b, m, l, LK_FULL), m, l, omega, loc, 0);
            loc ^= 1;
          }
        }
        loc0 ^= par;
      }
    }
    kb_update<DIM><<<grid, blk, 0, st>>>(I, full0, m, loc0);
  }
  for (int M = 2; M <= b->Mmax; ++M)
    launch_sweep_end<DIM>(M, grid, blk, st, I, Ls + list_sweep_m(b, M), reaction, b->d_rbits);
}

// Record one tick on the engine's stream (inside a capture): the lanes fork
// from it and join back before the residuals are read.  Lanes hold disjoint
// instances, so their only shared writes are atomic maxima into per-instance
// residual words and into the spread phase's scratch word.
template <int DIM>
void record_tick(isdc_batch* b, const Shape& sh) {
  cudaStream_t st = b->stream;
  cudaMemsetAsync(b->d_rbits, 0, sizeof(unsigned long long) * kMaxInst, st);
  if (sh.lanes > 1) {
    cudaEventRecord(b->ev_fork, st);
    for (int q = 1; q < sh.lanes; ++q) cudaStreamWaitEvent(b->lane_st[q - 1], b->ev_fork, 0);
  }
  for (int q = 0; q < sh.lanes; ++q) {
    cudaStream_t sq = q ? b->lane_st[q - 1] : st;
    if (sh.stagger && q > 0) cudaStreamWaitEvent(sq, b->ev_stage[q - 1], 0);
    record_lane<DIM>(b, sh, sq, b->d_lists + size_t(q) * b->nlists,
                     sh.stagger && q + 1 < sh.lanes ? b->ev_stage[q] : nullptr);
  }
  for (int q = 1; q < sh.lanes; ++q) {
    cudaEventRecord(b->ev_join[q - 1], b->lane_st[q - 1]);
    cudaStreamWaitEvent(st, b->ev_join[q - 1], 0);
  }
  cudaMemcpyAsync(b->h_rbits, b->d_rbits, sizeof(unsigned long long) * kMaxInst, cudaMemcpyDeviceToHost, st);
}

// The fused 2D tick as a phase table for the persistent launch: the same
// phases, lists and order as record_tick's fused mode.
isdc_status build_phases(isdc_batch* b) {
  if (b->d_phases) return ISDC_OK;
  std::vector<Phase> ph;
  auto add = [&](int kind, int list, int m, int l, int arg, int arg2) { ph.push_back(Phase{kind, list, m, l, arg, arg2}); };
  add(PH_SPREAD, list_spread(b), 0, 0, 0, 0);
  for (int M = 2; M <= b->Mmax; ++M) add(PH_SWEEP_END, list_spread_m(b, M), 0, 0, M, 0);
  const int Lg = bottom_level(2, b->max_side);
  for (int m = 0; m < b->Mmax - 1; ++m) {
    add(PH_RHS, list_index(b, m, 0, LK_FULL), m, 0, 0, 0);
    for (int c = 0; c < b->L; ++c) {
      for (int l = 0; l < Lg; ++l) add(PH_DOWN, list_index(b, m, l, LK_TILE), m, l, (l > 0 || c == 0) ? 1 : 0, 0);
      add(PH_BOTTOM, list_bottom(b, m), m, 0, c > 0 ? 1 : 0, 0);
      for (int l = Lg - 1; l >= 0; --l) add(PH_UP, list_index(b, m, l, LK_TILE), m, l, 0, 0);
    }
    add(PH_UPDATE, list_index(b, m, 0, LK_FULL), m, 0, 0, 0);
  }
  for (int M = 2; M <= b->Mmax; ++M) add(PH_SWEEP_END, list_sweep_m(b, M), 0, 0, M, 1);
  B_TRY(b, cudaMalloc(&b->d_phases, ph.size() * sizeof(Phase)));
  B_TRY(b, cudaMemcpy(b->d_phases, ph.data(), ph.size() * sizeof(Phase), cudaMemcpyHostToDevice));
  b->nphases = int(ph.size());
  return ISDC_OK;
}

// One tick as one cooperative launch; *unusable when the shape cannot be
// resident (the tuner then skips it).
isdc_status launch_persistent(isdc_batch* b, int shape, bool* unusable) {
  const Shape& sh = b->cands[shape];
  *unusable = false;
  isdc_status st = build_phases(b);
  if (st != ISDC_OK) return st;
  const void* fn = sh.threads == 512 ? reinterpret_cast<const void*>(kb_tick2<16>)
                   : sh.threads == 128 ? reinterpret_cast<const void*>(kb_tick2<4>)
                                       : reinterpret_cast<const void*>(kb_tick2<8>);
  const size_t smem = bottom_smem(2);
  if (b->pers_bps[shape] == 0) {
    int nb = 0;
    B_TRY(b, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    B_TRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.threads, smem));
    b->pers_bps[shape] = nb > 0 ? nb : -1;
  }
  if (b->pers_bps[shape] < 0) {
    *unusable = true;
    return ISDC_OK;
  }
  const dim3 grid(b->pers_bps[shape] * b->sms), blk(sh.threads);
  const Inst* insts = b->d_insts;
  const List* lists = b->d_lists;
  const Phase* phases = b->d_phases;
  int nph = b->nphases, reaction = b->opt.reaction, nu1 = b->opt.nu1, nu2 = b->opt.nu2;
  float omega = float(b->opt.omega);
  unsigned long long *rbits = b->d_rbits, *scratch = b->d_dummy;
  GridBarrier* gb = b->d_gb;
  void* args[] = {&insts, &lists, &phases, &nph, &reaction, &omega, &nu1, &nu2, &rbits, &scratch, &gb};
  B_TRY(b, cudaMemsetAsync(b->d_rbits, 0, sizeof(unsigned long long) * kMaxInst, b->stream));
  B_TRY(b, cudaMemsetAsync(b->d_gb, 0, sizeof(GridBarrier), b->stream));
  B_TRY(b, cudaLaunchCooperativeKernel(fn, grid, blk, args, smem, b->stream));
  B_TRY(b, cudaMemcpyAsync(b->h_rbits, b->d_rbits, sizeof(unsigned long long) * kMaxInst, cudaMemcpyDeviceToHost,
                           b->stream));
  B_TRY(b, cudaMemcpyAsync(b->h_gb, b->d_gb, sizeof(GridBarrier), cudaMemcpyDeviceToHost, b->stream));
  return ISDC_OK;
}

bool shape_allowed(const isdc_batch* b, int shape) {
  const Shape& sh = b->cands[shape];
  return !sh.persistent || tick_mode(b, sh) == MODE_FUSED2D;  // the persistent tick serves fused 2D only
}

// The autotuner has run every candidate so far: append the lane counts
// 2..kMaxLanes of the fastest graph shape (first time), else keep the fastest
// candidate for the engine's life.
void tuner_round_done(isdc_batch* b) {
  int best = 0;
  for (int s = 1; s < b->ncands; ++s)
    if (b->tune_rate[s] > b->tune_rate[best]) best = s;
  if (!b->lanes_added) {
    b->lanes_added = true;
    int g = -1;
    for (int s = 0; s < b->ncands; ++s)
      if (!b->cands[s].persistent && b->tune_rate[s] > 0.0 && (g < 0 || b->tune_rate[s] > b->tune_rate[g])) g = s;
    if (g >= 0) {
      for (int form = 0; form < 3; ++form)  // whole, split, split and staggered
        for (int q = 2; q <= kMaxLanes; ++q) {
          Shape sh = b->cands[g];
          sh.lanes = q;
          sh.split = form >= 1;
          sh.stagger = form == 2;
          b->cands[b->ncands++] = sh;
        }
      return;  // tune_next now points at the first lane candidate
    }
  }
  b->shape = best;
  b->tuned = 1;
}

isdc_status capture(isdc_batch* b, int shape) {
  if (b->exec[shape] || b->cands[shape].persistent) return ISDC_OK;
  cudaGraph_t g = nullptr;
  B_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  if (b->dim == 2) record_tick<2>(b, b->cands[shape]); else record_tick<3>(b, b->cands[shape]);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess) return bfail(b, ISDC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t q = 0; q < nn; ++q) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
          ++b->kernel_nodes[shape];
      }
  }
  e = cudaGraphInstantiate(&b->exec[shape], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, ISDC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return ISDC_OK;
}

void fill_instance(isdc_batch* b, int slot, int n, double nu, int M, double dt, unsigned char* mem) {
  Inst& I = b->h_insts[slot];
  std::memset(&I, 0, sizeof I);
  const int dim = b->dim;
  const size_t N = pts(dim, n);
  const double h = 1.0 / (n + 1);
  I.n = n;
  I.M = M;
  I.nlev = levels_of(n);
  I.lb = bottom_level(dim, n);
  I.nu_h2 = nu / (h * h);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    void* p = mem + off;
    off += align256(bytes);
    return p;
  };
  I.U = static_cast<double*>(take(size_t(M) * N * 8));
  I.F = static_cast<double*>(take(size_t(M) * N * 8));
  I.C = static_cast<double*>(take(size_t(M - 1) * N * 8));
  const bool jac = b->opt.smoother == ISDC_SMOOTHER_JACOBI;
  int side = n;
  for (int l = 0; l < I.nlev; ++l) {
    const size_t bytes = pts(dim, side) * 4;
    I.lev[l].n = side;
    I.lev[l].x = static_cast<float*>(take(bytes));
    I.lev[l].b = static_cast<float*>(take(bytes));
    I.lev[l].r = static_cast<float*>(take(bytes));
    I.lev[l].t = jac ? static_cast<float*>(take(bytes)) : nullptr;
    side = (side - 1) / 2;
  }
  I.ainv = static_cast<float*>(take(size_t(M - 1) * (dim == 2 ? 81 : 729) * 4));
  double tau[kMaxM], Q[kMaxM * kMaxM];
  host::lobatto_nodes(M, tau);
  host::q_matrix(M, tau, Q);
  for (int m = 0; m < M; ++m)
    for (int j = 0; j < M; ++j) I.dtQ[m][j] = dt * Q[m * M + j];
  for (int m = 0; m < M - 1; ++m) {
    I.dtm[m] = dt * (tau[m + 1] - tau[m]);
    const double a = I.dtm[m] * nu;
    int s = n;
    for (int l = 0; l < I.nlev; ++l) {
      const double hl = 1.0 / (s + 1), c = a / (hl * hl), d = 1.0 + 2.0 * dim * c;
      I.kappa[m][l] = float(c / d);
      if (l == 0) I.inv_d0[m] = 1.0 / d;
      if (l + 1 < I.nlev) {
        const int sc = (s - 1) / 2;
        const double hc = 1.0 / (sc + 1), cc = a / (hc * hc), dc = 1.0 + 2.0 * dim * cc;
        I.wscale[m][l] = float(d / (dc * (dim == 2 ? 16.0 : 64.0)));
      }
      s = (s - 1) / 2;
    }
  }
}

}  // namespace

ISDC_API isdc_status isdc_batch_create(int ndim, int64_t max_side, int max_M, size_t hbm_budget_bytes,
                                       int n_vcycles, const isdc_options* opt, isdc_batch** out) {
  if (!out) return bfail(nullptr, ISDC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return bfail(nullptr, ISDC_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (max_side < 7 || ((max_side + 1) & max_side) != 0 || (ndim == 3 && max_side > 1289) ||
      max_side > (int64_t(1) << (kMaxLevels + 1)) - 1)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "max_side must be 2^j - 1 >= 7 (got %lld)", (long long)max_side);
  if (max_M < 2 || max_M > kMaxM) return bfail(nullptr, ISDC_ERR_INVALID_ARG, "max_M must be in [2, %d]", kMaxM);
  if (n_vcycles < 1 || n_vcycles > 16) return bfail(nullptr, ISDC_ERR_INVALID_ARG, "n_vcycles must be in [1, 16]");
  isdc_options o;
  if (opt) o = *opt; else isdc_default_options(&o);
  if (o.smoother != ISDC_SMOOTHER_JACOBI && o.smoother != ISDC_SMOOTHER_RBGS)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "unknown smoother");
  if (o.use_graphs < 0 || o.use_graphs > 2)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "use_graphs must be 0, 1 or 2");
  if (o.smoother == ISDC_SMOOTHER_JACOBI && !(o.omega > 0 && o.omega <= 1))
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "the Jacobi damping omega must be in (0, 1]");
  if (o.nu1 < 1 || o.nu2 < 0 || o.nu1 > 8 || o.nu2 > 8)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "the batch engine needs 1 <= nu1 <= 8 and 0 <= nu2 <= 8");
  if (o.max_sweeps < 1) return bfail(nullptr, ISDC_ERR_INVALID_ARG, "max_sweeps must be >= 1");
  if (o.temporal_blocking < -1 || o.temporal_blocking > 1)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "the batch engine's temporal_blocking must be -1, 0 or 1");
  isdc_batch* b = new isdc_batch();
  b->dim = ndim;
  b->L = n_vcycles;
  b->Mmax = max_M;
  b->max_side = int(max_side);
  b->Lmax = levels_of(int(max_side));
  b->opt = o;
  b->opt.vcycle_fp32 = 1;
  // temporal-blocking depth of the 2D damped-Jacobi V(1, nu2 <= 1) cycles: 1 (the
  // default, option -1 or 1) fuses the sweep into the transfer passes, 0 keeps
  // separate phases; the two round differently, so the depth is fixed for the
  // engine's life
  b->fused = (ndim == 2 && o.smoother == ISDC_SMOOTHER_JACOBI && o.nu1 == 1 && o.nu2 <= 1 &&
              o.temporal_blocking != 0) ? 1 : 0;
  b->budget = hbm_budget_bytes;
  b->nlists = (max_M - 1) * b->Lmax * LK_KINDS + 2 * (max_M - 1) + 1 + 2 * (max_M - 1);
  auto bail = [&](isdc_status st) {
    snprintf(g_batch_error, sizeof g_batch_error, "%s", b->err);
    isdc_batch_destroy(b);
    return st;
  };
#define CB(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      bfail(b, e_ == cudaErrorMemoryAllocation ? ISDC_ERR_OOM : ISDC_ERR_CUDA, "%s: %s", #call, \
            cudaGetErrorString(e_));                                                    \
      return bail(e_ == cudaErrorMemoryAllocation ? ISDC_ERR_OOM : ISDC_ERR_CUDA);      \
    }                                                                                   \
  } while (0)
  int dev = 0;
  CB(cudaGetDevice(&dev));
  CB(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
  if (o.stream) {
    b->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    CB(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  CB(cudaMalloc(&b->d_insts, sizeof(Inst) * kMaxInst));
  CB(cudaMemset(b->d_insts, 0, sizeof(Inst) * kMaxInst));
  CB(cudaMallocHost(&b->h_insts, sizeof(Inst) * kMaxInst));
  CB(cudaMalloc(&b->d_lists, sizeof(List) * b->nlists * kMaxLanes));
  CB(cudaMallocHost(&b->h_lists, sizeof(List) * b->nlists * kMaxLanes));
  std::memset(b->h_lists, 0, sizeof(List) * b->nlists * kMaxLanes);
  CB(cudaMemset(b->d_lists, 0, sizeof(List) * b->nlists * kMaxLanes));
  CB(cudaMalloc(&b->d_rbits, sizeof(unsigned long long) * kMaxInst));
  CB(cudaMalloc(&b->d_dummy, sizeof(unsigned long long) * kMaxInst));
  CB(cudaMallocHost(&b->h_rbits, sizeof(unsigned long long) * kMaxInst));
  CB(cudaMalloc(&b->d_gb, sizeof(GridBarrier)));
  CB(cudaMallocHost(&b->h_gb, sizeof(GridBarrier)));
  std::memset(b->h_gb, 0, sizeof(GridBarrier));
  CB(cudaFuncSetAttribute(kb_bottom<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bottom_smem(2))));
  CB(cudaFuncSetAttribute(kb_bottom<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bottom_smem(3))));
  CB(cudaEventCreate(&b->ev0));
  CB(cudaEventCreate(&b->ev1));
  for (int q = 0; q < kMaxLanes - 1; ++q) {
    CB(cudaStreamCreateWithFlags(&b->lane_st[q], cudaStreamNonBlocking));
    CB(cudaEventCreateWithFlags(&b->ev_join[q], cudaEventDisableTiming));
    CB(cudaEventCreateWithFlags(&b->ev_stage[q], cudaEventDisableTiming));
  }
  CB(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  for (int q = 0; q < kNumBase; ++q) b->cands[q] = kBaseShapes[q];
  b->ncands = kNumBase;
#undef CB
  *out = b;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_batch_barrier_selftest(int blocks, int phantom, double limit_s, int* failed) {
  if (!failed || blocks < 1 || blocks > 1024 || phantom < 0 || phantom > 1024 || !(limit_s > 0.0 && limit_s <= 10.0))
    return bfail(nullptr, ISDC_ERR_INVALID_ARG,
                 "barrier self-test: 1 <= blocks <= 1024, 0 <= phantom <= 1024, 0 < limit_s <= 10");
  *failed = -1;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_barrier_selftest, 32, 0);
  if (e != cudaSuccess) return bfail(nullptr, ISDC_ERR_CUDA, "barrier self-test: %s", cudaGetErrorString(e));
  if (blocks > sms * per_sm)
    return bfail(nullptr, ISDC_ERR_INVALID_ARG, "barrier self-test: %d blocks cannot all be resident", blocks);
  GridBarrier* d = nullptr;
  GridBarrier h{};
  e = cudaMalloc(&d, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(GridBarrier));
  if (e == cudaSuccess) {
    unsigned int ph = unsigned(phantom);
    unsigned long long ns = (unsigned long long)(limit_s * 1e9);
    void* args[] = {&d, &ph, &ns};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kb_barrier_selftest), dim3(blocks), dim3(32), args,
                                    0, nullptr);
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(GridBarrier), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(nullptr, ISDC_ERR_CUDA, "barrier self-test: %s", cudaGetErrorString(e));
  *failed = h.err ? 1 : 0;
  return ISDC_OK;
}

ISDC_API void isdc_batch_destroy(isdc_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int i = 0; i < kMaxInst; ++i)
    if (b->slots[i].mem) cudaFreeAsync(b->slots[i].mem, b->stream);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int s = 0; s < kMaxCands; ++s)
    if (b->exec[s]) cudaGraphExecDestroy(b->exec[s]);
  for (int q = 0; q < kMaxLanes - 1; ++q) {
    if (b->lane_st[q]) cudaStreamDestroy(b->lane_st[q]);
    if (b->ev_join[q]) cudaEventDestroy(b->ev_join[q]);
    if (b->ev_stage[q]) cudaEventDestroy(b->ev_stage[q]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  cudaFree(b->d_insts);
  cudaFreeHost(b->h_insts);
  cudaFree(b->d_lists);
  cudaFreeHost(b->h_lists);
  cudaFree(b->d_rbits);
  cudaFree(b->d_dummy);
  cudaFreeHost(b->h_rbits);
  cudaFree(b->d_gb);
  cudaFreeHost(b->h_gb);
  cudaFree(b->d_phases);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

ISDC_API isdc_status isdc_batch_admit(isdc_batch* b, const isdc_problem* p, const double* u0, int u0_on_host,
                                      int* slot_out) {
  if (!b || !p || !u0 || !slot_out) return ISDC_ERR_INVALID_ARG;
  *slot_out = -1;
  const int64_t n = p->n;
  if (n < 7 || n > b->max_side || ((n + 1) & n) != 0)
    return bfail(b, ISDC_ERR_INVALID_ARG, "side must be 2^j - 1 in [7, %d] (got %lld)", b->max_side, (long long)n);
  if (p->M < 2 || p->M > b->Mmax) return bfail(b, ISDC_ERR_INVALID_ARG, "M must be in [2, %d]", b->Mmax);
  if (!(p->nu > 0) || !(p->dt > 0) || !std::isfinite(p->nu) || !std::isfinite(p->dt) || p->steps < 1)
    return bfail(b, ISDC_ERR_INVALID_ARG, "need nu > 0, dt > 0, steps >= 1");
  int slot = -1;
  for (int i = 0; i < kMaxInst; ++i)
    if (b->slots[i].state == ISDC_SLOT_FREE) { slot = i; break; }
  if (slot < 0) return bfail(b, ISDC_ERR_OOM, "all %d slots are in use", kMaxInst);
  const size_t bytes = instance_bytes(b, int(n), p->M);
  if (b->used + bytes > b->budget)
    return bfail(b, ISDC_ERR_OOM, "instance needs %zu bytes; %zu of %zu budget bytes in use", bytes, b->used,
                 b->budget);
  void* mem = nullptr;
  B_TRY(b, cudaMallocAsync(&mem, bytes, b->stream));
  fill_instance(b, slot, int(n), p->nu, p->M, p->dt, static_cast<unsigned char*>(mem));
  Inst& I = b->h_insts[slot];
  const size_t N = pts(b->dim, int(n));
  // initial value goes to the last node: a step's spread starts from u_{M-1}
  B_TRY(b, cudaMemcpyAsync(I.U + size_t(p->M - 1) * N, u0, N * 8,
                           u0_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->stream));
  std::vector<float> ainv(size_t(p->M - 1) * (b->dim == 2 ? 81 : 729));
  for (int m = 0; m < p->M - 1; ++m) {
    std::vector<double> inv;
    const double a = I.dtm[m] * p->nu;
    host::coarse_inverse(b->dim, a, inv);
    const double d3 = 1.0 + 2.0 * b->dim * a * 16.0;
    for (size_t q = 0; q < inv.size(); ++q) ainv[m * inv.size() + q] = float(d3 * inv[q]);
  }
  B_TRY(b, cudaMemcpyAsync(I.ainv, ainv.data(), ainv.size() * 4, cudaMemcpyHostToDevice, b->stream));
  B_TRY(b, cudaMemcpyAsync(b->d_insts + slot, &b->h_insts[slot], sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
  B_TRY(b, cudaStreamSynchronize(b->stream));  // the host staging (ainv, pinned descriptor) is reused
  Slot& S = b->slots[slot];
  S = Slot();
  S.state = ISDC_SLOT_RUNNING;
  S.n = int(n);
  S.M = p->M;
  S.nlev = levels_of(int(n));
  S.steps = p->steps;
  S.spread_next = true;
  S.bytes = bytes;
  S.mem = mem;
  b->used += bytes;
  *slot_out = slot;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_batch_tick(isdc_batch* b, int* running_out, int* finished_out) {
  if (!b) return ISDC_ERR_INVALID_ARG;
  int running = 0;
  double dofs = 0.0;
  for (int i = 0; i < kMaxInst; ++i)
    if (b->slots[i].state == ISDC_SLOT_RUNNING) {
      ++running;
      dofs += double(pts(b->dim, b->slots[i].n));
    }
  int finished = 0;
  if (running) {
    // the persistent shapes serve the fused 2D mode only; the tuner skips them otherwise
    for (;;) {
      while (!b->tuned && b->tune_next < b->ncands && !shape_allowed(b, b->tune_next))
        b->tune_rate[b->tune_next++] = 0.0;
      if (b->tuned || b->tune_next < b->ncands) break;
      tuner_round_done(b);
    }
    int shape = b->tuned ? b->shape : b->tune_next;
    isdc_status st = capture(b, shape);
    if (st != ISDC_OK) return st;
    auto upload_lists = [&](const Shape& sh) -> isdc_status {
      build_lists(b, sh);
      B_TRY(b, cudaMemcpyAsync(b->d_lists, b->h_lists, sizeof(List) * b->nlists * sh.lanes, cudaMemcpyHostToDevice,
                               b->stream));
      return ISDC_OK;
    };
    if ((st = upload_lists(b->cands[shape])) != ISDC_OK) return st;
    b->last_tick_bytes = tick_bytes(b, b->cands[shape]);
    B_TRY(b, cudaEventRecord(b->ev0, b->stream));
    bool skip = false;
    const int tried = shape;
    if (b->cands[shape].persistent) {
      if ((st = launch_persistent(b, shape, &skip)) != ISDC_OK) return st;
      if (skip) {  // cannot be resident: take the first graph shape for this tick
        shape = 0;
        if ((st = capture(b, shape)) != ISDC_OK) return st;
        if ((st = upload_lists(b->cands[shape])) != ISDC_OK) return st;
      } else {
        b->kernel_launches += 1;
      }
    }
    if (!b->cands[shape].persistent) {
      B_TRY(b, cudaGraphLaunch(b->exec[shape], b->stream));
      b->kernel_launches += b->kernel_nodes[shape];
    }
    B_TRY(b, cudaEventRecord(b->ev1, b->stream));
    B_TRY(b, cudaStreamSynchronize(b->stream));
    if (b->cands[shape].persistent && b->h_gb->err)
      return bfail(b, ISDC_ERR_CUDA, "a grid barrier of the persistent tick waited longer than its limit");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    if (!b->tuned && !b->tune_warm) {
      b->tune_warm = true;  // warm-up tick: not scored, the same shape is tried again next tick
    } else if (!b->tuned) {  // autotuner: one real tick per candidate, keep the fastest
      b->tune_rate[tried] = skip ? 0.0 : dofs / std::max(ms, 1e-3f);
      if (++b->tune_next == b->ncands) tuner_round_done(b);
    }
    ++b->ticks;
    for (int i = 0; i < kMaxInst; ++i) {
      Slot& S = b->slots[i];
      if (S.state != ISDC_SLOT_RUNNING) continue;
      double R;
      std::memcpy(&R, &b->h_rbits[i], sizeof R);
      S.spread_next = false;
      S.sweeps += 1;
      S.total_sweeps += 1;
      S.last_res = R;
      if (!std::isfinite(R)) {
        S.state = ISDC_SLOT_FAILED;
        ++finished;
        continue;
      }
      const bool conv = R < b->opt.tol;
      if (conv || S.sweeps >= b->opt.max_sweeps) {
        if (!conv) ++S.nonconverged;
        S.steps_done += 1;
        S.sweeps = 0;
        if (S.steps_done >= S.steps) {
          S.state = ISDC_SLOT_FINISHED;
          ++finished;
        } else {
          S.spread_next = true;
        }
      }
    }
  }
  if (running_out) {
    int r = 0;
    for (int i = 0; i < kMaxInst; ++i) r += b->slots[i].state == ISDC_SLOT_RUNNING;
    *running_out = r;
  }
  if (finished_out) *finished_out = finished;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_batch_query(const isdc_batch* b, int slot, isdc_slot_info* info) {
  if (!b || !info || slot < 0 || slot >= kMaxInst) return ISDC_ERR_INVALID_ARG;
  const Slot& S = b->slots[slot];
  info->state = S.state;
  info->steps_done = S.steps_done;
  info->sweeps_in_step = S.sweeps;
  info->total_sweeps = S.total_sweeps;
  info->nonconverged_steps = S.nonconverged;
  info->last_residual = S.last_res;
  info->device_bytes = S.bytes;
  return ISDC_OK;
}

ISDC_API isdc_status isdc_batch_take(isdc_batch* b, int slot, double* u_out, int out_on_host) {
  if (!b || slot < 0 || slot >= kMaxInst) return ISDC_ERR_INVALID_ARG;
  Slot& S = b->slots[slot];
  if (S.state == ISDC_SLOT_FREE) return bfail(b, ISDC_ERR_INVALID_ARG, "slot %d is free", slot);
  if (S.state == ISDC_SLOT_RUNNING && u_out)
    return bfail(b, ISDC_ERR_INVALID_ARG, "slot %d is still running", slot);
  if (u_out) {
    const Inst& I = b->h_insts[slot];
    const size_t N = pts(b->dim, S.n);
    B_TRY(b, cudaMemcpyAsync(u_out, I.U + size_t(S.M - 1) * N, N * 8,
                             out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
  }
  B_TRY(b, cudaFreeAsync(S.mem, b->stream));
  B_TRY(b, cudaStreamSynchronize(b->stream));
  b->used -= S.bytes;
  S = Slot();
  return ISDC_OK;
}

ISDC_API isdc_status isdc_batch_stats(const isdc_batch* b, isdc_batch_info* info) {
  if (!b || !info) return ISDC_ERR_INVALID_ARG;
  info->ticks = b->ticks;
  info->kernel_launches = b->kernel_launches;
  info->bytes_in_use = b->used;
  info->tuned = b->tuned;
  const Shape& cur = b->cands[b->tuned ? b->shape : b->tune_next % b->ncands];
  info->threads_per_block = cur.threads;
  info->blocks_per_sm = cur.blocks_per_sm;
  info->fused = tick_mode(b, cur) == MODE_FUSED2D;
  info->lanes = cur.lanes;
  info->lane_split = cur.split + cur.stagger;
  {
    const int sh = b->tuned ? b->shape : b->tune_next % b->ncands;
    info->kernels_per_tick = b->cands[sh].persistent ? 1 : b->kernel_nodes[sh];
    if (b->cands[sh].persistent) info->blocks_per_sm = b->pers_bps[sh];
  }
  info->bytes_last_tick = b->last_tick_bytes;
  int r = 0;
  for (int i = 0; i < kMaxInst; ++i) r += b->slots[i].state == ISDC_SLOT_RUNNING;
  info->running = r;
  return ISDC_OK;
}

ISDC_API const char* isdc_batch_last_error(const isdc_batch* b) { return b ? b->err : g_batch_error; }
