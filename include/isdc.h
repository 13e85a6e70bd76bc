/*
 * isdc.h -- C ABI of the GB300 (sm_103a) implementation of inexact spectral
 * deferred corrections (ISDC; Speck, Ruprecht, Minion, Emmett, Krause,
 * arXiv:1401.7824).
 *
 * Problem (Sec. 2, Eq. 1): u(t) = u_0 + int_{T_0}^t f(u(s)) ds with
 *   f(u) = f^I(u) + f^E(u),  f^I(u) = A u,  A = nu * L_h,
 * L_h the 5-point (2D) or 7-point (3D) Laplacian on the interior points of the
 * unit square/cube with zero Dirichlet values (Sec. 3, the linearly implicit
 * case with W = I), and f^E(u) = u - u^3 or 0 (explicit part of Eq. 4).
 *
 * One time step [T_n, T_n + dt] runs semi-implicit SDC sweeps (Sec. 2, Eq. 4)
 * over M Gauss-Lobatto nodes; every implicit Euler solve
 * (I - dt_m A) u_{m+1}^{k+1} = rhs is replaced by L geometric-multigrid
 * V-cycles started from u_{m+1}^k (Sec. 3, Sec. 4.3).  Sweeps stop when the
 * max-norm SDC residual (Sec. 3) drops below a tolerance, or after a fixed
 * count.
 *
 * Layout of every grid array: float64, interior points only, x fastest:
 * index i + n*(j + n*k) for 0-based i, j, k in [0, n).  h = 1/(n+1).
 *
 * Conventions:
 *  - Device pointers are CUDA global-memory pointers valid on the device that
 *    was current when the context was created.  The caller owns every buffer
 *    it passes; the library never frees or keeps them past the call.
 *  - Work is ordered on the context's stream.  Calls that return host values
 *    (isdc_residual, isdc_stats, isdc_step with n_sweeps = 0, isdc_step_host)
 *    synchronise that stream.
 *  - Errors are return codes; nothing aborts or traps.  isdc_last_error()
 *    describes the last failure.  A context is not thread-safe; separate
 *    contexts are independent.
 */
#ifndef ISDC_H
#define ISDC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isdc_ctx isdc_ctx;

typedef enum {
    ISDC_OK = 0,
    ISDC_ERR_INVALID_ARG = 1,   /* bad size, parameter or NULL pointer            */
    ISDC_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement   */
    ISDC_ERR_OOM = 3,           /* device allocation failed                       */
    ISDC_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed    */
    ISDC_ERR_NOT_CONVERGED = 5, /* soft: max_sweeps reached; u holds the last sweep */
    ISDC_ERR_NONFINITE = 6,     /* the SDC residual became NaN or Inf             */
    ISDC_ERR_SCRATCH_TOO_SMALL = 7 /* isdc_vcycles_static: the grid's multigrid buffers do not
                                      fit in its static scratch array                  */
} isdc_status;

/* Collocation node families (Sec. 2: t_0 = T_n <= t_1 < ... < t_M <= T_{n+1}).
 * Gauss-Lobatto: tau_1 = 0, tau_M = 1, t_0 is node 1, M-1 node solves per sweep.
 * Gauss-Radau (right): tau_M = 1, M node solves per sweep from t_0.
 * Gauss-Legendre: interior nodes, M node solves per sweep, and the step ends
 * with the full-step quadrature u_{n+1} = u_0 + dt sum_j w_j f(u_j). */
typedef enum {
    ISDC_NODES_GAUSS_LOBATTO = 0,
    ISDC_NODES_RADAU_RIGHT = 1,
    ISDC_NODES_GAUSS_LEGENDRE = 2
} isdc_node_type;

typedef enum { ISDC_SMOOTHER_JACOBI = 0, ISDC_SMOOTHER_RBGS = 1 } isdc_smoother;
typedef enum { ISDC_REACTION_NONE = 0, ISDC_REACTION_ALLEN_CAHN = 1 } isdc_reaction;

typedef struct {
    int    smoother;      /* isdc_smoother: damped Jacobi (default) or red-black Gauss-Seidel */
    int    nu1, nu2;      /* pre/post smoothing sweeps per level (default 1, 1) */
    double omega;         /* Jacobi damping (default 2/3; must lie in (0, 1] with the Jacobi smoother) */
    int    vcycle_fp32;   /* 0: V-cycles in FP64.  1: FP32 V-cycles in defect-correction
                             form (FP64 defect b - (I - dt_m A)x, FP32 cycle on the error,
                             FP64 update); node values, S F, residuals stay FP64. */
    int    reaction;      /* isdc_reaction (default ISDC_REACTION_ALLEN_CAHN) */
    double tol;           /* SDC residual tolerance for n_sweeps == 0 (default 1e-10) */
    int    max_sweeps;    /* sweep cap for n_sweeps == 0 (default 100) */
    double mg_tol;        /* classical SDC (n_vcycles == 0): stop the node solve when the
                             max-norm residual of (I - dt_m A)x = b is <= mg_tol (default 1e-12) */
    int    mg_max_cycles; /* cap on V-cycles per node solve in that mode (default 50) */
    int    vcycle_cap;    /* 0 (default): n_vcycles = L > 0 runs exactly L V-cycles.  1: L is a
                             cap and a node solve stops early once its max-norm residual is
                             <= mg_tol (one residual check, and host synchronisation, per cycle) */
    int    use_graphs;    /* 1 (default): a sweep with a fixed V-cycle count is captured once as a
                             CUDA graph and replayed (same kernels, same order), each kernel
                             launched as soon as every block of the one before it has started and
                             waiting at entry for that kernel to complete (programmatic
                             dependencies); 2: the same graph with ordinary dependencies; 0:
                             launch one by one.  Every choice gives the same result bit for bit.
                             With the profiler on, the graph carries its event nodes and the
                             stream is synchronised after every replay to read them. */
    int    temporal_blocking; /* 3D, FP32 V-cycles, red-black: smoothing of the fine level.
                             -1 (default): chosen by the autotuner in isdc_create.  0: one pass
                             over the grid per colour.  1 or 2: that many complete red-black
                             sweeps per pass over HBM (temporal blocking; the same FP32
                             operations in the same order, so the same result bit for bit).
                             Other configurations ignore it. */
    int    stencil;       /* 0 (default): 5-point (2D) / 7-point (3D) Laplacian, W = I.
                             1: the 4th-order compact 9-point Laplacian with the weighting
                             matrix W of Sec. 3 (Eq. 5), 2D, damped-Jacobi smoothing, FP64
                             V-cycles (other combinations: ISDC_ERR_UNSUPPORTED). */
    int    equation;      /* 0 (default): u_t = nu Lap u + f^E(u) on the unit square / cube, zero
                             Dirichlet values, sides 2^j - 1 (interior points), h = 1/(n+1).
                             1: viscous Burgers u_t + sum_axes u u_x = nu Lap u (Sec. 4.1) on the
                             periodic [-1,1)^ndim, sides 2^j with j >= 3, h = 2/n; the advection is
                             explicit (5th-order WENO, local Lax-Friedrichs splitting), the
                             Laplacian implicit (periodic multigrid); FP64 V-cycles; `reaction`
                             is ignored. */
    int    rb_run;        /* 3D red-black smoothing of the natural-layout levels (launch shape, not
                             from the paper): 0 (default) lets the autotuner in isdc_create pick,
                             per level, the points each thread updates along a diagonal run and how
                             it issues them; 1, 2, 4, 8, 16 or 32: runs of that many points with
                             the next point's loads issued before each store; -1, -2, -4 or -8:
                             runs of that many points with all loads issued first.  Every choice
                             gives the same result bit for bit. */
    int    fused_transfer; /* residual + full-weighting restriction on every level above the
                             single-block bottom (launch form, not from the paper): -1 (default)
                             lets the autotuner in isdc_create time both forms per level and keep
                             the faster; 1: one launch, the fine residual kept in shared memory;
                             0: two launches, the residual written to device memory and read
                             back.  Every choice gives the same result bit for bit. */
    void  *stream;        /* cudaStream_t to run on.  NULL: the context creates its own
                             non-blocking stream.  To run on the legacy default stream pass
                             cudaStreamLegacy ((void*)1), for the per-thread default stream
                             cudaStreamPerThread ((void*)2). */
} isdc_options;

/* Fill *opt with the defaults listed above.  Returns ISDC_ERR_INVALID_ARG for NULL. */
isdc_status isdc_default_options(isdc_options *opt);

/*
 * Collocation tables of Sec. 2 (Eq. 2) on the unit interval, host only (no
 * GPU needed): nodes tau[M] (ascending; tau_1 = 0, tau_M = 1 for
 * Gauss-Lobatto), the integration matrix Q[M*M] (Q[m*M+j] = integral from 0 to
 * tau_m of the Lagrange basis polynomial l_j over the nodes) and, if S is not
 * NULL, the matrix of the sweep's steps between consecutive points
 * t_0 <= t_1 < ... : S[R*M] with R = M-1 rows (Gauss-Lobatto, S_m = Q_{m+1} -
 * Q_m) or R = M rows (Radau, Legendre: S_0 = Q_1, S_m = Q_{m+1} - Q_m).  The
 * S_m^{m+1} F(u) of Eq. 2 is dt * sum_j S[m*M+j] f(u_j).
 * Errors: INVALID_ARG (node type, M outside [2, 7], NULL tau or Q).
 */
isdc_status isdc_collocation_tables(isdc_node_type nodes, int M, double *tau, double *Q, double *S);

/*
 * Create a context for one problem: the collocation tables (Sec. 2, Eq. 2:
 * nodes tau_m, Q, S_m^{m+1}, dt_m = t_{m+1} - t_m), the device node state
 * (u and f(u) at t_0 and every node) and the multigrid hierarchy (sides
 * n, (n-1)/2, ... down to 3).
 *   ndim   2 or 3
 *   dims   ndim sides, all equal: 2^j - 1 interior points with 2 <= j <= 13 (equation 0) or
 *          2^j periodic points with 3 <= j <= 13 (equation 1), so that the hierarchy has at
 *          most 12 levels; 3D sides at most 1289 (32-bit point indices)
 *   nu     diffusion coefficient (> 0)
 *   nodes  isdc_node_type (Gauss-Lobatto, Gauss-Radau right or Gauss-Legendre)
 *   M      number of nodes, 2..7
 *   dt     time-step length (> 0)
 *   opt    options, or NULL for the defaults
 *   out    receives the context (NULL on failure)
 * Allocates device memory (cudaMalloc) on the current device.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
isdc_status isdc_create(int ndim, const int64_t *dims, double nu, isdc_node_type nodes, int M,
                        double dt, const isdc_options *opt, isdc_ctx **out);

/*
 * Advance u by one time step (Sec. 2, Eq. 4; Sec. 3).
 *   u          device pointer, N = n^ndim float64 values; on entry u(T_n), on
 *              return u(T_n + dt): u_M (Gauss-Lobatto, Radau: tau_M = 1) or
 *              u_0 + dt sum_j w_j f(u_j) (Gauss-Legendre)
 *   n_sweeps   > 0: exactly that many sweeps (no host synchronisation);
 *              0: sweep until the SDC residual < opt.tol, at most opt.max_sweeps
 *   n_vcycles  L > 0: L V-cycles per node solve (ISDC);
 *              0: classical SDC, V-cycles until the node residual <= opt.mg_tol
 * The multigrid initial guess is always u_{m+1}^k (Sec. 4.3).  The initial
 * iterate is u spread to all nodes, unless isdc_set_nodes() supplied one.
 * Errors: INVALID_ARG, CUDA, NOT_CONVERGED (soft, u holds the last sweep),
 * NONFINITE.
 */
isdc_status isdc_step(isdc_ctx *ctx, double *u, int n_sweeps, int n_vcycles);

/*
 * isdc_step for a HOST buffer: copies u (N float64 in host memory, pinned or
 * pageable) to the device, runs the step, copies the result back and
 * synchronises.  Same arguments and errors as isdc_step.
 */
isdc_status isdc_step_host(isdc_ctx *ctx, double *u_host, int n_sweeps, int n_vcycles);

/* Max-norm SDC residual after the last sweep of the last step (Sec. 3), to
 * *res (host).  Synchronises.  Errors: INVALID_ARG, CUDA. */
isdc_status isdc_residual(const isdc_ctx *ctx, double *res);

/* Sweeps and V-cycles (node solves only) spent by the last step, to host
 * pointers (either may be NULL).  Synchronises. */
isdc_status isdc_stats(const isdc_ctx *ctx, int *sweeps, int64_t *vcycles);

/* Residual after each sweep of the last step: copies min(cap, sweeps) values
 * to hist (host) and the sweep count to *count.  Only filled in the
 * until-tolerance mode (n_sweeps == 0) and in fixed mode with record = 1 in
 * isdc_set_record_history(). */
isdc_status isdc_residual_history(const isdc_ctx *ctx, double *hist, int cap, int *count);

/* Record the residual of every sweep in fixed-sweep mode too (one device-to-
 * host copy per sweep, no extra synchronisation until the step ends). */
isdc_status isdc_set_record_history(isdc_ctx *ctx, int record);

/* Copy the M node values u_1..u_M of the last sweep (M*N float64, node-major)
 * to the device buffer dst.  Checkpoint / inspection. */
isdc_status isdc_get_nodes(const isdc_ctx *ctx, double *dst);

/* Use the M*N node values in the device buffer src as the initial iterate of
 * the NEXT isdc_step instead of spreading u (resume from a checkpoint).  With
 * Gauss-Lobatto nodes the first node must equal that step's u; with the other
 * families t_0 is not a node and takes that step's u.  Applies to one step only. */
isdc_status isdc_set_nodes(isdc_ctx *ctx, const double *src);

/*
 * Standalone multigrid solve on one implicit Euler system of Sec. 3,
 * (I - a L_h) x = b, with the context's grid and smoother: n_cycles V-cycles
 * from the initial x (FP64 or FP32 per opt.vcycle_fp32).  x, b: device, N
 * float64 each; x is updated in place.  Uses the context's hierarchy.
 */
isdc_status isdc_vcycles(isdc_ctx *ctx, double a, double *x, const double *b, int n_cycles);

/*
 * isdc_vcycles_static -- the same multigrid solve as isdc_vcycles, for callers
 * that cannot allocate device memory.  (The paper has no counterpart; this is
 * an interface for integrators.)  Examples: code running under another
 * framework's memory manager that has already reserved the device memory,
 * real-time loops that must never call cudaMalloc, or code that must not
 * allocate while other work is being captured into a CUDA graph.
 *
 * Runs n_cycles V-cycles (FP64) on (I - a L_h) x = b on the ndim-dimensional
 * grid of side n (2^j - 1), with the given smoother (ISDC_SMOOTHER_*), nu1/nu2
 * sweeps and Jacobi damping omega, on 'stream' (a cudaStream_t; NULL is the
 * legacy default stream).  x, b: device, n^ndim float64 each, x updated in
 * place; the caller owns both.  Asynchronous on the stream.
 *
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The
 * coarse grids, the fine-grid residual (and Jacobi) buffers, the scaled
 * right-hand side and the side-3 inverse live in one static device array of ISDC_STATIC_SCRATCH_BYTES that
 * every GPU which loads this library keeps until the process exits.  Grids
 * whose buffers exceed it (2D sides above 1023, 3D sides above 127) are
 * rejected with ISDC_ERR_SCRATCH_TOO_SMALL before any GPU work.  With the
 * Jacobi smoother omega must lie in (0, 1] (else INVALID_ARG).
 *
 * The first call on each device (with that device current) looks up the
 * array's device address and sets the bottom kernels' shared-memory limit;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents (everything a call needs is
 * rewritten by that call), so calls that overlap on the GPU -- on different
 * streams or from different host threads -- race and must not be issued.
 * Errors: INVALID_ARG, SCRATCH_TOO_SMALL, UNSUPPORTED, CUDA.
 */
#define ISDC_STATIC_SCRATCH_BYTES (64u << 20)
isdc_status isdc_vcycles_static(int ndim, int64_t n, double a, int smoother, int nu1, int nu2, double omega,
                                double *x, const double *b, int n_cycles, void *stream);

/*
 * Batched and continuously batched integration (not from the paper: the
 * serving layer around it).  An engine holds up to 256 independent ISDC
 * integrations of one dimension (each with its own side, nu, M, dt and number
 * of time steps; the smoother, nu1/nu2, L, tol and max_sweeps are the
 * engine's).  Every tick advances every running instance by one SDC sweep:
 * each phase of the sweep is one grid-stride launch over all instances taking
 * part, and the whole tick is one CUDA graph.  The coarse levels of every
 * instance (2D sides <= 63, 3D sides <= 15) run in one block per instance in
 * shared memory; with 2D damped-Jacobi V(1, nu2 <= 1) cycles the sweep of each
 * grid-wide level is fused into its transfer passes (one pass per leg and
 * level).  V-cycles run in FP32 in
 * defect-correction form; node values, S F, node residuals and the SDC
 * residual are FP64.  Instances are admitted and their results taken between
 * ticks; device memory for an instance is taken with cudaMallocAsync on
 * admission, within the engine's HBM budget, and returned by isdc_batch_take.
 * An engine is not thread-safe.
 */
typedef struct isdc_batch isdc_batch;

typedef struct {
    int64_t n;     /* interior side, 2^j - 1, 7 <= n <= the engine's max_side */
    double  nu;    /* diffusion coefficient */
    int     M;     /* Gauss-Lobatto nodes, 2 <= M <= the engine's max_M */
    double  dt;    /* time-step length */
    int     steps; /* time steps to run */
} isdc_problem;

enum { ISDC_SLOT_FREE = 0, ISDC_SLOT_RUNNING = 1, ISDC_SLOT_FINISHED = 2, ISDC_SLOT_FAILED = 3 };

typedef struct {
    int     state;              /* ISDC_SLOT_* */
    int     steps_done;
    int     sweeps_in_step;     /* sweeps of the current step so far */
    int     total_sweeps;
    int     nonconverged_steps; /* steps that ended at max_sweeps without reaching tol */
    double  last_residual;      /* SDC residual after the instance's last sweep */
    size_t  device_bytes;       /* device memory held by the instance */
} isdc_slot_info;

typedef struct {
    int64_t ticks;
    int64_t kernel_launches;    /* kernels executed by all ticks (kernel nodes of the tick graphs) */
    size_t  bytes_in_use;
    int     running;
    int     tuned;              /* 1 once the autotuner has picked the launch shape */
    int     threads_per_block;  /* launch shape in use (tile = one point per thread; the fused 2D
                                   phases' tile is 32 x threads/32 coarse points, the red-black
                                   phases' tile threads/32 grid rows) */
    int     blocks_per_sm;      /* persistent blocks per SM */
    int     fused;              /* 1: the 2D damped-Jacobi smoother is fused into the transfer
                                   passes (one pass per leg and level); 0: separate phases */
    int     kernels_per_tick;   /* kernel launches of one tick in the shape in use */
    double  bytes_last_tick;    /* algorithmic device-memory bytes of the last tick (each phase
                                   reads each input once and writes each output once) */
    int     lanes;              /* independent chains of the tick graph in use, each over its own
                                   share of the running instances (run concurrently) */
    int     lane_split;         /* 1: each lane's launches take blocks_per_sm / lanes blocks per SM,
                                   so the lanes' blocks share the SMs; 2: the same, and lane q
                                   starts once lane q-1's first right-hand side is done (lanes a
                                   phase apart); 0: all blocks_per_sm */
} isdc_batch_info;

/* ndim 2 or 3; max_side: the largest side that will be admitted (sets the
 * number of multigrid phases; 2^j - 1 with 3 <= j <= 13, in 3D at most 1289); max_M <= 7; hbm_budget_bytes: device memory the
 * instances may hold together; n_vcycles: L >= 1; opt as for isdc_create
 * (nu1 >= 1 is required; vcycle_fp32 is implied; stream NULL = own stream;
 * temporal_blocking for 2D damped-Jacobi V(1, nu2 <= 1) engines: -1 or 1 fuse
 * the sweep into the transfer passes, 0 keeps it a separate phase; other
 * values INVALID_ARG; the two round differently, so the choice is fixed for
 * the engine's life; use_graphs must be 0, 1 or 2 but is not used: a tick is
 * always one graph launch with ordinary dependencies or, in 2D fused mode, one
 * cooperative launch).  The first ticks try several launch shapes (tile size,
 * blocks per SM, one launch per tick, then 1 to 4 lanes: concurrent chains of
 * the tick graph over disjoint shares of the instances, each with all or
 * 1/lanes of the blocks per SM, the latter also staggered by a phase; all give
 * the same result bit for bit) and keep the fastest (autotuner).
 * Errors: INVALID_ARG, OOM, CUDA. */
isdc_status isdc_batch_create(int ndim, int64_t max_side, int max_M, size_t hbm_budget_bytes, int n_vcycles,
                              const isdc_options *opt, isdc_batch **out);

/* Admit one integration with initial value u0 (n^ndim float64; host memory if
 * u0_on_host, else device).  *slot receives the instance's slot.  Returns
 * ISDC_ERR_OOM (soft: retry after taking results) when the budget or the
 * slots are exhausted.  Synchronises the engine's stream. */
isdc_status isdc_batch_admit(isdc_batch *b, const isdc_problem *p, const double *u0, int u0_on_host, int *slot);

/* One sweep for every running instance (one graph launch); synchronises.
 * *running: instances still running afterwards; *finished: instances that
 * finished (or failed) in this tick.  Either pointer may be NULL. */
isdc_status isdc_batch_tick(isdc_batch *b, int *running, int *finished);

isdc_status isdc_batch_query(const isdc_batch *b, int slot, isdc_slot_info *info);

/* Copy a finished instance's solution (u after its last step; n^ndim float64,
 * host memory if out_on_host, else device; u_out may be NULL to discard) and
 * free its slot and device memory. */
isdc_status isdc_batch_take(isdc_batch *b, int slot, double *u_out, int out_on_host);

isdc_status isdc_batch_stats(const isdc_batch *b, isdc_batch_info *info);

/* Message for the last failure of b, or of isdc_batch_create when b is NULL. */
const char *isdc_batch_last_error(const isdc_batch *b);

void isdc_batch_destroy(isdc_batch *b);

/* Self-test of the bounded grid barrier of the one-launch batch tick (no
 * paper counterpart; failure detection).  One cooperative launch of `blocks`
 * blocks (all resident) runs two barrier rounds that expect `phantom` more
 * arrivals than there are blocks.  *failed = 0 when both rounds complete
 * (phantom = 0), 1 when a wait ran out after limit_s seconds; in that case
 * every block sets the error flag and returns, the kernel ends normally and
 * the device stays usable.  Synchronises the device.
 * Errors: INVALID_ARG (blocks outside [1, 1024] or more than can be resident,
 * phantom outside [0, 1024], limit_s outside (0, 10], failed NULL; checked
 * before any device work except the occupancy query), CUDA. */
isdc_status isdc_batch_barrier_selftest(int blocks, int phantom, double limit_s, int *failed);

/* Per-kernel-class timing (not from the paper: instrumentation for the
 * roofline).  While enabled, every launch of the context is bracketed by CUDA
 * events on its stream, and the algorithmic bytes and floating-point
 * operations of the launch (a model: every input read once, every output
 * written once; one op = one add, multiply or fused multiply-add) are summed.
 * Enabling resets the sums. */
typedef struct {
    char    name[32];   /* kernel class, e.g. "smooth_fine", "sweep_end" */
    int64_t launches;
    double  total_ms;   /* sum of event-timed launch durations; -1 if the class was not timed */
    double  bytes;      /* algorithmic bytes, summed over launches */
    double  fp64_ops;   /* algorithmic FP64 operations, summed */
    double  fp32_ops;   /* algorithmic FP32 operations, summed */
} isdc_kernel_stat;

/* enable = 0: off.  Otherwise a bit mask over the kernel classes, in this
 * order: spread, eval_f, rhs, sweep_end, smooth_fine, residual_fine,
 * restrict_fine, prolong_fine, smooth_coarse, residual_coarse,
 * restrict_coarse, prolong_coarse, bottom, defect, update, resnorm, w_inverse
 * (bit 0 = spread).  Launch counts, bytes and ops are kept for every class;
 * only the classes in the mask get events (-1 times them all).  A value with
 * no class bit but another bit set (e.g. 1 << 30) counts launches, bytes and
 * ops without events and without the per-sweep synchronisation that reading
 * graph-replayed events needs. */
isdc_status isdc_profile_enable(isdc_ctx *ctx, int enable);

/* Synchronise and copy up to cap class records (classes with launches only)
 * to out; *count receives the number of such classes. */
isdc_status isdc_profile_read(isdc_ctx *ctx, isdc_kernel_stat *out, int cap, int *count);

/* Launch shape chosen by the context's autotuner (not from the paper): points
 * per thread of the fine-level red-black smoother in FP64 (the length of the
 * thread's diagonal run) and in FP32 (z-planes per thread of the split level);
 * 3D red-black contexts time 1 to 32 points (1 to 8 planes on the split level)
 * on their own arrays in isdc_create, otherwise 1; for the FP32 fine level also the temporal-blocking depth
 * (red-black sweeps per pass, 0 = one pass per colour) and the z-planes per
 * block of the blocked pass.  Any output pointer may be NULL. */
isdc_status isdc_tuning(const isdc_ctx *ctx, int *zb_fp64, int *zb_fp32, int *tb_depth, int *tb_planes);

/* The residual + restriction form chosen for each grid-wide multigrid level
 * l = 0 .. *n_levels - 1 (the levels above the single-block bottom; 0 for the
 * compact-stencil and periodic configurations): kc[l] = 0 two launches,
 * kc[l] > 0 one fused launch (3D: kc[l] coarse planes per block).  Fills at
 * most max_levels entries of kc (host); n_levels may be NULL.
 * Errors: INVALID_ARG. */
isdc_status isdc_tuning_transfer(const isdc_ctx *ctx, int *kc, int max_levels, int *n_levels);

/* Message for the last failure of ctx, or of isdc_create when ctx is NULL. */
const char *isdc_last_error(const isdc_ctx *ctx);

/* Free the context and its device memory (synchronises its stream). */
void isdc_destroy(isdc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ISDC_H */
