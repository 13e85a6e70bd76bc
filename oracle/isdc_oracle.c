/*
 * isdc_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for
 * inexact spectral deferred corrections (Speck, Ruprecht, Minion, Emmett,
 * Krause, "Inexact spectral deferred corrections", arXiv:1401.7824).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may import, call, link or execute
 * anything under oracle/.  The product path (the CUDA library) never does, and
 * this file shares no code, header, table or helper with it.
 *
 * What it computes, step by step in the paper's order and notation:
 *   - collocation nodes tau_1 < ... < tau_M in [0,1] (Sec. 2 names
 *     Gauss-Lobatto and Gauss-Legendre; Gauss-Radau with tau_M = 1 as well):
 *     t_0 = T_n <= t_1 < ... < t_M <= T_{n+1}, and the integration matrices
 *     Q (Q[m][j] = int_0^{tau_m} l_j) and S (point-to-point,
 *     S_m^{m+1} = Q_{m+1} - Q_m, with the row of t_0 zero)    -- Sec. 2, Eq. 2
 *   - the semi-implicit SDC sweep                             -- Sec. 2, Eq. 4
 *       u_{m+1}^{k+1} = u_m^{k+1} + dt_m[f^I(u_{m+1}^{k+1}) - f^I(u_{m+1}^k)]
 *                     + dt_m[f^E(u_m^{k+1}) - f^E(u_m^k)] + S_m^{m+1}F(u^k)
 *     with f^I(u) = A u, A = nu * L_h (5-point 2D / 7-point 3D Laplacian,
 *     zero Dirichlet ghosts, W = I in Eq. 5), and f^E(u) = u - u^3
 *     (or none, or lambda_E*u for the Dahlquist order test);
 *   - or, in 2D, the 4th-order compact discretisation of Sec. 3: the 9-point
 *     Laplacian L_9 with the weighting matrix W = I + (h^2/12) L_5, so that
 *     W u' = nu L_9 u + W f^E(u), f^I = W^{-1} nu L_9, and the sweep of Eq. 5
 *       (W - dt_m A) u_{m+1}^{k+1} = W u_m^{k+1} + dt_m W[f^E(u_m^{k+1}) - f^E(u_m^k)]
 *                                  - dt_m A u_{m+1}^k + S_m^{m+1} F~(u^k)
 *     with A = nu L_9 and f~ = W f^E + A u; the SDC residual inverts W once
 *     per node (exactly, by the sine transform);
 *   - each implicit Euler solve (I - dt_m A) x = b done either exactly
 *     (sine-transform diagonalisation: classical SDC with an exact spatial
 *     solve, Sec. 3), by multigrid until a tolerance (classical SDC, Sec. 3),
 *     or by L fixed V-cycles started from u_{m+1}^k (ISDC, Sec. 3 and Sec. 4.3);
 *   - the max-norm SDC residual after every sweep               -- Sec. 3;
 *   - or the viscous Burgers equation of Sec. 4.1 on a periodic grid: the
 *     Laplacian implicit (periodic 5/7-point), the advection sum_axes (u^2/2)_x
 *     explicit with the 5th-order WENO finite-difference scheme of Jiang and
 *     Shu (local Lax-Friedrichs flux splitting), periodic multigrid and an
 *     exact solve by the discrete Fourier transform.
 *
 * The multigrid solver is not described in the paper (Acknowledgments); the
 * one here is textbook geometric multigrid: vertex-centred coarsening
 * n_c = (n-1)/2 down to side 3, rediscretised coarse operators I - a L_{2h},
 * full-weighting restriction, (bi/tri)linear prolongation, one recursive call
 * per level (V-cycle), zero coarse initial guess, exact dense solve on the
 * side-3 grid, and either damped Jacobi or red-black Gauss-Seidel smoothing.
 *
 * Threads: built once plainly (the pragmas below are ignored) and once with
 * -fopenmp for the all-core variant.  Only the outermost grid loops of the
 * stencil, transfer, solve and pointwise steps carry a pragma (each iteration
 * writes its own points; a red-black colour reads only the other colour), and
 * the max-norms combine per-thread maxima (max is exact in any order), so both
 * builds give the same results bit for bit.
 *
 * Grid layout: interior points only, x fastest.  With 1-based interior
 * indices i,j,k in 1..n the array index is (i-1) + n*((j-1) + n*(k-1)).
 * h = 1/(n+1).  Everything is IEEE double, built with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_M 16

/* ------------------------------------------------------------------------ */
/* Problem description passed from Python (ctypes mirrors this layout).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int    ndim;        /* 2 or 3 */
    int    n;           /* interior points per side, 2^j - 1 */
    double nu;          /* diffusion coefficient in f^I = nu L_h u */
    int    M;           /* number of Gauss-Lobatto nodes, 2..ORC_MAX_M */
    double dt;          /* time step Delta t */
    int    reaction;    /* f^E: 0 none, 1 u - u^3, 2 lambda_e * u */
    double lambda_e;    /* coefficient for reaction 2 */
    int    smoother;    /* 0 damped Jacobi, 1 red-black Gauss-Seidel */
    int    nu1, nu2;    /* pre- and post-smoothing sweeps */
    double omega;       /* Jacobi damping */
    int    solver;      /* 0 ISDC: L V-cycles; 1 classical: MG until mg_tol;
                           2 classical: exact sine-transform solve;
                           3 ISDC with L as a cap: at most L V-cycles, stopping
                             early once the node residual is <= mg_tol */
    int    guess;       /* multigrid start: 0 u_{m+1}^k (Sec. 4.3), 1 zero,
                           2 u_m^{k+1} */
    double tol;         /* SDC residual tolerance */
    int    max_sweeps;  /* cap for the until-tolerance mode */
    double mg_tol;      /* classical SDC: max-norm residual of the node solve */
    int    mg_max_cycles;
    int    nodes;       /* 0 Gauss-Lobatto, 1 Gauss-Radau (right, tau_M = 1),
                           2 Gauss-Legendre */
    int    stencil;     /* 0: 5-point (2D) / 7-point (3D) Laplacian, W = I;
                           1: 4th-order compact 9-point Laplacian with the
                           weighting matrix W (Sec. 3, Eq. 5), 2D only */
    int    equation;    /* 0: u_t = nu Lap u + f^E(u) on the unit square/cube with
                           zero Dirichlet values (n = 2^j - 1 interior points);
                           1: viscous Burgers u_t + sum_axes u u_x = nu Lap u on
                           the periodic [-1,1)^d (n = 2^j points, h = 2/n),
                           advection explicit by 5th-order WENO (Sec. 4.1) */
} orc_problem;

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and quadrature nodes (Sec. 2: collocation nodes).   */
/* ------------------------------------------------------------------------ */

/* P_n(x) and P_n'(x) on [-1,1] by the three-term recurrence. */
static void legendre(int n, double x, double *p, double *dp)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    *p = p1;
    /* (x^2 - 1) P_n'(x) = n (x P_n - P_{n-1}) */
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre nodes/weights on [-1,1]: roots of P_n by Newton. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(n, z, &p, &dp);
            double dz = p / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p, dp;
        legendre(n, z, &p, &dp);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/*
 * Gauss-Lobatto nodes on [0,1]: the end points plus the roots of P'_{M-1}
 * mapped from [-1,1].  The roots of P'_{M-1} are found by Newton's method on
 * P'_{M-1}, using P''_{M-1} from the Legendre ODE
 * (1-x^2) P'' = 2x P' - n(n+1) P.
 */
int orc_lobatto_nodes(int M, double *tau)
{
    if (M < 2 || M > ORC_MAX_M) return 1;
    int n = M - 1;
    double z[ORC_MAX_M];
    z[0] = -1.0;
    z[M - 1] = 1.0;
    for (int i = 1; i < M - 1; ++i) {
        double x = -cos(M_PI * i / n); /* Chebyshev-Lobatto start */
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(n, x, &p, &dp);
            double d2p = (2.0 * x * dp - n * (n + 1.0) * p) / (1.0 - x * x);
            double dx = dp / d2p;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        z[i] = x;
    }
    for (int i = 0; i < M; ++i) tau[i] = 0.5 * (z[i] + 1.0);
    tau[0] = 0.0;
    tau[M - 1] = 1.0;
    return 0;
}

/*
 * Right Gauss-Radau nodes on [0,1]: the M roots of P_M - P_{M-1} on [-1,1]
 * (x = 1 is one of them), mapped to [0,1].  The roots are bracketed by sign
 * changes on a fine uniform grid of [-1,1) and refined by bisection.
 */
int orc_radau_right_nodes(int M, double *tau)
{
    if (M < 2 || M > ORC_MAX_M) return 1;
    const int samples = 4000 * M;
    int found = 0;
    double a = -1.0, pa, pb, dp;
    legendre(M, a, &pa, &dp);
    legendre(M - 1, a, &pb, &dp);
    double ga = pa - pb;
    for (int s = 1; s < samples && found < M - 1; ++s) {
        double b = -1.0 + 2.0 * s / samples;
        legendre(M, b, &pa, &dp);
        legendre(M - 1, b, &pb, &dp);
        double gb = pa - pb;
        if ((ga < 0.0) != (gb < 0.0)) {
            double lo = a, hi = b, glo = ga;
            for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
                double mid = 0.5 * (lo + hi), pm, pm1;
                legendre(M, mid, &pm, &dp);
                legendre(M - 1, mid, &pm1, &dp);
                double gm = pm - pm1;
                if ((gm < 0.0) == (glo < 0.0)) { lo = mid; glo = gm; } else hi = mid;
            }
            tau[found++] = 0.5 * (0.5 * (lo + hi) + 1.0);
        }
        a = b;
        ga = gb;
    }
    if (found != M - 1) return 2;
    tau[M - 1] = 1.0;
    return 0;
}

/* Gauss-Legendre nodes on [0,1]: the roots of P_M mapped from [-1,1], ascending. */
int orc_legendre_nodes(int M, double *tau)
{
    if (M < 1 || M > ORC_MAX_M) return 1;
    double x[ORC_MAX_M], w[ORC_MAX_M];
    gauss_legendre(M, x, w);
    /* gauss_legendre returns them in descending order (cosine start values) */
    for (int i = 0; i < M; ++i) tau[i] = 0.5 * (x[M - 1 - i] + 1.0);
    return 0;
}

/* Nodes of the given family (0 Lobatto, 1 Radau right, 2 Legendre). */
int orc_nodes(int kind, int M, double *tau)
{
    if (kind == 0) return orc_lobatto_nodes(M, tau);
    if (kind == 1) return orc_radau_right_nodes(M, tau);
    if (kind == 2) return orc_legendre_nodes(M, tau);
    return 1;
}

/* Lagrange basis polynomial l_j over the nodes tau, evaluated at s. */
static double lagrange(int M, const double *tau, int j, double s)
{
    double v = 1.0;
    for (int i = 0; i < M; ++i)
        if (i != j) v *= (s - tau[i]) / (tau[j] - tau[i]);
    return v;
}

/*
 * Q[m][j] = int_0^{tau_m} l_j(s) ds (row-major, M x M).  l_j has degree M-1,
 * so an M-point Gauss-Legendre rule on [0, tau_m] integrates it exactly.
 */
int orc_q_matrix(int M, const double *tau, double *Q)
{
    if (M < 2 || M > ORC_MAX_M) return 1;
    double gx[ORC_MAX_M], gw[ORC_MAX_M];
    gauss_legendre(M, gx, gw);
    for (int m = 0; m < M; ++m) {
        double half = 0.5 * tau[m];
        for (int j = 0; j < M; ++j) {
            double acc = 0.0;
            for (int g = 0; g < M; ++g)
                acc += gw[g] * lagrange(M, tau, j, half * (gx[g] + 1.0));
            Q[m * M + j] = half * acc;
        }
    }
    return 0;
}

/* Full-interval weights w_j = int_0^1 l_j(s) ds (the end-point quadrature of
 * the collocation rule; with tau_M = 1 they are the last row of Q). */
int orc_end_weights(int M, const double *tau, double *w)
{
    if (M < 1 || M > ORC_MAX_M) return 1;
    double gx[ORC_MAX_M], gw[ORC_MAX_M];
    gauss_legendre(M, gx, gw);
    for (int j = 0; j < M; ++j) {
        double acc = 0.0;
        for (int g = 0; g < M; ++g) acc += gw[g] * lagrange(M, tau, j, 0.5 * (gx[g] + 1.0));
        w[j] = 0.5 * acc;
    }
    return 0;
}

/* S_m^{m+1} = Q_{m+1} - Q_m, m = 0..M-2 (rows of an (M-1) x M matrix). Eq. 2 */
int orc_s_matrix(int M, const double *Q, double *S)
{
    if (M < 2 || M > ORC_MAX_M) return 1;
    for (int m = 0; m < M - 1; ++m)
        for (int j = 0; j < M; ++j)
            S[m * M + j] = Q[(m + 1) * M + j] - Q[m * M + j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers.                                                             */
/* ------------------------------------------------------------------------ */
static long npoints(int d, int n) { return d == 2 ? (long)n * n : (long)n * n * n; }

static long idx(int d, int n, int i, int j, int k)
{
    if (d == 2) return (i - 1) + (long)n * (j - 1);
    return (i - 1) + (long)n * ((j - 1) + (long)n * (k - 1));
}

/* Value at 1-based interior index; zero on (or beyond) the Dirichlet boundary. */
static double val(const double *u, int d, int n, int i, int j, int k)
{
    if (i < 1 || i > n || j < 1 || j > n) return 0.0;
    if (d == 3 && (k < 1 || k > n)) return 0.0;
    return u[idx(d, n, i, j, k)];
}

static int kmax(int d, int n) { return d == 3 ? n : 1; }

/* Sum of the 2d nearest neighbours of (i,j,k). */
static double neighbour_sum(const double *u, int d, int n, int i, int j, int k)
{
    double s = val(u, d, n, i - 1, j, k) + val(u, d, n, i + 1, j, k)
             + val(u, d, n, i, j - 1, k) + val(u, d, n, i, j + 1, k);
    if (d == 3) s += val(u, d, n, i, j, k - 1) + val(u, d, n, i, j, k + 1);
    return s;
}

/* L_h u at one point: (sum of neighbours - 2d u) / h^2. */
static double laplacian_at(const double *u, int d, int n, int i, int j, int k)
{
    double h = 1.0 / (n + 1);
    return (neighbour_sum(u, d, n, i, j, k) - 2.0 * d * val(u, d, n, i, j, k)) / (h * h);
}

/* out = L_h u (5-point in 2D, 7-point in 3D). */
void orc_laplacian(int d, int n, const double *u, double *out)
{
    const int km = kmax(d, n);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k <= km; ++k)
        for (int j = 1; j <= n; ++j)
            for (int i = 1; i <= n; ++i)
                out[idx(d, n, i, j, k)] = laplacian_at(u, d, n, i, j, k);
}

/* r = b - (I - a L_h) x */
void orc_residual(int d, int n, double a, const double *x, const double *b, double *r)
{
    const int km = kmax(d, n);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k <= km; ++k)
        for (int j = 1; j <= n; ++j)
            for (int i = 1; i <= n; ++i) {
                long p = idx(d, n, i, j, k);
                r[p] = b[p] - (x[p] - a * laplacian_at(x, d, n, i, j, k));
            }
}

/* max_p |v_p| */
static double max_abs(const double *v, long N)
{
    double m = 0.0;
#pragma omp parallel
    {
        double mt = 0.0;
#pragma omp for schedule(static) nowait
        for (long p = 0; p < N; ++p) {
            double a = fabs(v[p]);
            if (a > mt || a != a) mt = a; /* a NaN propagates */
        }
#pragma omp critical
        if (mt > m || mt != mt) m = mt;
    }
    return m;
}

/* Plain copy of N values (the threaded build splits it over the cores). */
static void copy_values(double *dst, const double *src, long N)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) dst[p] = src[p];
}

/* Threads for the loops of the threaded build (no effect in the plain build). */
void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Number of threads the oracle's loops use (1 in the plain build). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Multigrid components.                                                     */
/* ------------------------------------------------------------------------ */

/*
 * One damped-Jacobi sweep on (I - a L_h) x = b:
 *   x_new = x_old + omega (b - (I - a L_h) x_old) / (1 + 2 d a / h^2),
 * every point from the old iterate.  'old' is scratch of N values.
 */
void orc_smooth_jacobi(int d, int n, double a, double omega, double *x, const double *b,
                       double *old)
{
    double h = 1.0 / (n + 1);
    double diag = 1.0 + 2.0 * d * a / (h * h);
    copy_values(old, x, npoints(d, n));
    const int km = kmax(d, n);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k <= km; ++k)
        for (int j = 1; j <= n; ++j)
            for (int i = 1; i <= n; ++i) {
                long p = idx(d, n, i, j, k);
                double r = b[p] - (old[p] - a * laplacian_at(old, d, n, i, j, k));
                x[p] = old[p] + omega * r / diag;
            }
}

/*
 * One red-black Gauss-Seidel sweep on (I - a L_h) x = b.  A point is red when
 * i+j(+k) is even (1-based interior indices); all red points are relaxed
 * first, then all black points, each solving its own row exactly:
 *   x_p = (b_p + (a/h^2) * sum of neighbours) / (1 + 2 d a / h^2).
 */
void orc_smooth_rbgs(int d, int n, double a, double *x, const double *b)
{
    double h = 1.0 / (n + 1);
    double diag = 1.0 + 2.0 * d * a / (h * h);
    const int km = kmax(d, n);
    for (int colour = 0; colour < 2; ++colour)
#pragma omp parallel for collapse(2) schedule(static)
        for (int k = 1; k <= km; ++k)
            for (int j = 1; j <= n; ++j)
                for (int i = 1; i <= n; ++i) {
                    int parity = (d == 3) ? (i + j + k) % 2 : (i + j) % 2;
                    if (parity != colour) continue;
                    long p = idx(d, n, i, j, k);
                    x[p] = (b[p] + a * neighbour_sum(x, d, n, i, j, k) / (h * h)) / diag;
                }
}

/* 1D full-weighting / linear-interpolation weight between fine i and coarse I. */
static double hat(int i, int I)
{
    int off = i - 2 * I;
    if (off == 0) return 1.0;
    if (off == 1 || off == -1) return 0.5;
    return 0.0;
}

/*
 * Full-weighting restriction from the fine grid (side n) to the coarse grid
 * (side nc = (n-1)/2).  Coarse point I sits on fine point 2I; weights are the
 * tensor product of (1/4, 1/2, 1/4): 1/16 [1 2 1; 2 4 2; 1 2 1] in 2D, /64 in 3D.
 */
void orc_restrict_fw(int d, int n, const double *r, double *rc)
{
    int nc = (n - 1) / 2;
    const int Km = kmax(d, nc);
#pragma omp parallel for collapse(2) schedule(static)
    for (int K = 1; K <= Km; ++K)
        for (int J = 1; J <= nc; ++J)
            for (int I = 1; I <= nc; ++I) {
                double acc = 0.0;
                int kc = (d == 3) ? 2 * K : 1;
                int klo = (d == 3) ? kc - 1 : 1, khi = (d == 3) ? kc + 1 : 1;
                for (int k = klo; k <= khi; ++k)
                    for (int j = 2 * J - 1; j <= 2 * J + 1; ++j)
                        for (int i = 2 * I - 1; i <= 2 * I + 1; ++i) {
                            double w = 0.5 * hat(i, I) * 0.5 * hat(j, J);
                            if (d == 3) w *= 0.5 * hat(k, K);
                            acc += w * val(r, d, n, i, j, k);
                        }
                rc[idx(d, nc, I, J, K)] = acc;
            }
}

/*
 * x += P e_c with P the (bi/tri)linear interpolation from the coarse grid
 * (side nc) to the fine grid (side n = 2 nc + 1); coarse values beyond the
 * interior are the zero Dirichlet ghosts.
 */
void orc_prolong_add(int d, int nc, const double *ec, double *x)
{
    int n = 2 * nc + 1;
    const int km = kmax(d, n);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k <= km; ++k)
        for (int j = 1; j <= n; ++j)
            for (int i = 1; i <= n; ++i) {
                double acc = 0.0;
                int Klo = (d == 3) ? k / 2 : 1, Khi = (d == 3) ? (k + 1) / 2 : 1;
                for (int K = Klo; K <= Khi; ++K)
                    for (int J = j / 2; J <= (j + 1) / 2; ++J)
                        for (int I = i / 2; I <= (i + 1) / 2; ++I) {
                            double w = hat(i, I) * hat(j, J);
                            if (d == 3) w *= hat(k, K);
                            acc += w * val(ec, d, nc, I, J, K);
                        }
                x[idx(d, n, i, j, k)] += acc;
            }
}

/* ------------------------------------------------------------------------ */
/* 4th-order compact discretisation (Sec. 3), 2D only.                       */
/* ------------------------------------------------------------------------ */

/* Sum of the 4 corner (diagonal) neighbours of (i,j); zero outside. */
static double corner_sum(const double *u, int n, int i, int j)
{
    return val(u, 2, n, i - 1, j - 1, 1) + val(u, 2, n, i + 1, j - 1, 1)
         + val(u, 2, n, i - 1, j + 1, 1) + val(u, 2, n, i + 1, j + 1, 1);
}

/* L_9 u = (4 * edge neighbours + corner neighbours - 20 u) / (6 h^2) */
static double lap9_at(const double *u, int n, int i, int j)
{
    double h = 1.0 / (n + 1);
    return (4.0 * neighbour_sum(u, 2, n, i, j, 1) + corner_sum(u, n, i, j) - 20.0 * val(u, 2, n, i, j, 1))
           / (6.0 * h * h);
}

/* W u = u + (h^2/12) L_5 u = (8 u + edge neighbours) / 12 */
static double w_at(const double *u, int n, int i, int j)
{
    return (8.0 * val(u, 2, n, i, j, 1) + neighbour_sum(u, 2, n, i, j, 1)) / 12.0;
}

/* out = L_9 u */
void orc_laplacian9(int n, const double *u, double *out)
{
    for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) out[idx(2, n, i, j, 1)] = lap9_at(u, n, i, j);
}

/* out = W u */
void orc_apply_w(int n, const double *u, double *out)
{
    for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) out[idx(2, n, i, j, 1)] = w_at(u, n, i, j);
}

/* r = b - (W - a L_9) x */
void orc_residual9(int n, double a, const double *x, const double *b, double *r)
{
    for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) {
            long p = idx(2, n, i, j, 1);
            r[p] = b[p] - (w_at(x, n, i, j) - a * lap9_at(x, n, i, j));
        }
}

/*
 * One damped-Jacobi sweep on (W - a L_9) x = b: every point from the old
 * iterate, x += omega (b - (W - a L_9) x_old) / diag, diag = 8/12 + 20 a/(6 h^2).
 */
void orc_smooth_jacobi9(int n, double a, double omega, double *x, const double *b, double *old)
{
    double h = 1.0 / (n + 1);
    double diag = 8.0 / 12.0 + 20.0 * a / (6.0 * h * h);
    memcpy(old, x, sizeof(double) * npoints(2, n));
    for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) {
            long p = idx(2, n, i, j, 1);
            double r = b[p] - (w_at(old, n, i, j) - a * lap9_at(old, n, i, j));
            x[p] = old[p] + omega * r / diag;
        }
}

void orc_residual_per(int d, int n, double a, const double *x, const double *b, double *r);

/*
 * Exact solve on a small grid: the dense matrix of the operator (I - a L_h for
 * stencil 0, W - a L_9 for stencil 1, periodic I - a L_h for 2) assembled column by column by applying
 * it to unit vectors, then Gaussian elimination with partial pivoting.  Used
 * on the coarsest multigrid level.
 */
static void dense_solve(int stencil, int d, int n, double a, const double *b, double *x)
{
    long N = npoints(d, n);
    double *A = (double *)malloc(sizeof(double) * N * N);
    double *e = (double *)calloc(N, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * N);
    double *rhs = (double *)malloc(sizeof(double) * N);
    double *zero = (double *)calloc(N, sizeof(double));
    for (long c = 0; c < N; ++c) {
        e[c] = 1.0;
        /* column c of the operator = -(residual of x = e with b = 0) */
        if (stencil == 1) orc_residual9(n, a, e, zero, col);
        else if (stencil == 2) orc_residual_per(d, n, a, e, zero, col);
        else orc_residual(d, n, a, e, zero, col);
        for (long r = 0; r < N; ++r) A[r * N + c] = -col[r];
        e[c] = 0.0;
    }
    for (long r = 0; r < N; ++r) rhs[r] = b[r];
    for (long c = 0; c < N; ++c) {
        long piv = c;
        for (long r = c + 1; r < N; ++r)
            if (fabs(A[r * N + c]) > fabs(A[piv * N + c])) piv = r;
        if (piv != c) {
            for (long q = 0; q < N; ++q) {
                double t = A[c * N + q]; A[c * N + q] = A[piv * N + q]; A[piv * N + q] = t;
            }
            double t = rhs[c]; rhs[c] = rhs[piv]; rhs[piv] = t;
        }
        for (long r = c + 1; r < N; ++r) {
            double f = A[r * N + c] / A[c * N + c];
            for (long q = c; q < N; ++q) A[r * N + q] -= f * A[c * N + q];
            rhs[r] -= f * rhs[c];
        }
    }
    for (long r = N - 1; r >= 0; --r) {
        double s = rhs[r];
        for (long q = r + 1; q < N; ++q) s -= A[r * N + q] * x[q];
        x[r] = s / A[r * N + r];
    }
    free(A); free(e); free(col); free(rhs); free(zero);
}

void orc_dense_solve(int d, int n, double a, const double *b, double *x) { dense_solve(0, d, n, a, b, x); }
void orc_dense_solve9(int n, double a, const double *b, double *x) { dense_solve(1, 2, n, a, b, x); }

/* ------------------------------------------------------------------------ */
/* Periodic grids (viscous Burgers, Sec. 4.1): n points per side with        */
/* 0-based indices i = 0..n-1 at x_i = -1 + i h, h = 2/n, wrapping around.   */
/* ------------------------------------------------------------------------ */
static long pidx(int d, int n, int i, int j, int k)
{
    i = ((i % n) + n) % n;
    j = ((j % n) + n) % n;
    if (d == 2) return i + (long)n * j;
    k = ((k % n) + n) % n;
    return i + (long)n * (j + (long)n * k);
}

static double pnsum(const double *u, int d, int n, int i, int j, int k)
{
    double s = u[pidx(d, n, i - 1, j, k)] + u[pidx(d, n, i + 1, j, k)]
             + u[pidx(d, n, i, j - 1, k)] + u[pidx(d, n, i, j + 1, k)];
    if (d == 3) s += u[pidx(d, n, i, j, k - 1)] + u[pidx(d, n, i, j, k + 1)];
    return s;
}

/* periodic L_h u at (i,j,k), h = 2/n */
static double plap_at(const double *u, int d, int n, int i, int j, int k)
{
    double h = 2.0 / n;
    return (pnsum(u, d, n, i, j, k) - 2.0 * d * u[pidx(d, n, i, j, k)]) / (h * h);
}

static int pkmax(int d, int n) { return d == 3 ? n : 1; }

void orc_laplacian_per(int d, int n, const double *u, double *out)
{
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) out[pidx(d, n, i, j, k)] = plap_at(u, d, n, i, j, k);
}

/* r = b - (I - a L_h) x, periodic */
void orc_residual_per(int d, int n, double a, const double *x, const double *b, double *r)
{
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                long p = pidx(d, n, i, j, k);
                r[p] = b[p] - (x[p] - a * plap_at(x, d, n, i, j, k));
            }
}

void orc_smooth_jacobi_per(int d, int n, double a, double omega, double *x, const double *b, double *old)
{
    double h = 2.0 / n, diag = 1.0 + 2.0 * d * a / (h * h);
    memcpy(old, x, sizeof(double) * npoints(d, n));
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                long p = pidx(d, n, i, j, k);
                double r = b[p] - (old[p] - a * plap_at(old, d, n, i, j, k));
                x[p] = old[p] + omega * r / diag;
            }
}

/* red-black Gauss-Seidel, red = i+j(+k) even (0-based); n even keeps the
 * colouring consistent across the wrap-around */
void orc_smooth_rbgs_per(int d, int n, double a, double *x, const double *b)
{
    double h = 2.0 / n, diag = 1.0 + 2.0 * d * a / (h * h);
    for (int colour = 0; colour < 2; ++colour)
        for (int k = 0; k < pkmax(d, n); ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    int parity = (d == 3) ? (i + j + k) % 2 : (i + j) % 2;
                    if (parity != colour) continue;
                    long p = pidx(d, n, i, j, k);
                    x[p] = (b[p] + a * pnsum(x, d, n, i, j, k) / (h * h)) / diag;
                }
}

/* full weighting to the coarse periodic grid (n/2 points): coarse I sits on
 * fine 2I, weights (1/4, 1/2, 1/4) per axis, wrapping around */
void orc_restrict_per(int d, int n, const double *r, double *rc)
{
    int nc = n / 2;
    for (int K = 0; K < pkmax(d, nc); ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                double acc = 0.0;
                for (int dk = (d == 3 ? -1 : 0); dk <= (d == 3 ? 1 : 0); ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            double w = (di ? 0.25 : 0.5) * (dj ? 0.25 : 0.5);
                            if (d == 3) w *= dk ? 0.25 : 0.5;
                            acc += w * r[pidx(d, n, 2 * I + di, 2 * J + dj, 2 * K + dk)];
                        }
                rc[pidx(d, nc, I, J, K)] = acc;
            }
}

/* x += P e_c: linear interpolation from the coarse periodic grid */
void orc_prolong_per(int d, int nc, const double *ec, double *x)
{
    int n = 2 * nc;
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                /* fine i lies on coarse i/2 (even) or between (i-1)/2 and (i+1)/2 (odd) */
                for (int K = (d == 3 ? k / 2 : 0); K <= (d == 3 ? (k + 1) / 2 : 0); ++K)
                    for (int J = j / 2; J <= (j + 1) / 2; ++J)
                        for (int I = i / 2; I <= (i + 1) / 2; ++I) {
                            double w = (i % 2 ? 0.5 : (I * 2 == i ? 1.0 : 0.0))
                                     * (j % 2 ? 0.5 : (J * 2 == j ? 1.0 : 0.0));
                            if (d == 3) w *= k % 2 ? 0.5 : (K * 2 == k ? 1.0 : 0.0);
                            acc += w * ec[pidx(d, nc, I, J, K)];
                        }
                x[pidx(d, n, i, j, k)] += acc;
            }
}

/*
 * Exact solve of (I - a L_h) x = b on the periodic grid by the discrete
 * Fourier transform: the modes exp(2 pi i (p i' + q j' [+ r k'])/n) are
 * eigenvectors of L_h with eigenvalues -(4/h^2) sum_axes sin^2(pi p/n).  The
 * transforms are dense complex sums along each axis.
 */
static void dft_along_axis(int d, int n, int axis, double *re, double *im, int sign)
{
    long N = npoints(d, n), st = 1;
    for (int a = 0; a < axis; ++a) st *= n;
    double *lr = (double *)malloc(sizeof(double) * n), *li = (double *)malloc(sizeof(double) * n);
    for (long base = 0; base < N; ++base) {
        if ((base / st) % n != 0) continue;
        for (int p = 0; p < n; ++p) {
            double ar = 0.0, ai = 0.0;
            for (int q = 0; q < n; ++q) {
                double ang = sign * 2.0 * M_PI * (double)p * (double)q / n;
                double c = cos(ang), s = sin(ang);
                double xr = re[base + q * st], xi = im[base + q * st];
                ar += xr * c - xi * s;
                ai += xr * s + xi * c;
            }
            lr[p] = ar;
            li[p] = ai;
        }
        for (int p = 0; p < n; ++p) { re[base + p * st] = lr[p]; im[base + p * st] = li[p]; }
    }
    free(lr); free(li);
}

void orc_solve_exact_per(int d, int n, double a, const double *b, double *x)
{
    long N = npoints(d, n);
    double h = 2.0 / n;
    double *re = (double *)malloc(sizeof(double) * N), *im = (double *)calloc(N, sizeof(double));
    memcpy(re, b, sizeof(double) * N);
    for (int ax = 0; ax < d; ++ax) dft_along_axis(d, n, ax, re, im, -1);
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double si = sin(M_PI * i / n), sj = sin(M_PI * j / n), sk = d == 3 ? sin(M_PI * k / n) : 0.0;
                double lam = -4.0 * (si * si + sj * sj + sk * sk) / (h * h);
                long p = pidx(d, n, i, j, k);
                double f = 1.0 / ((1.0 - a * lam) * (double)N);
                re[p] *= f;
                im[p] *= f;
            }
    for (int ax = 0; ax < d; ++ax) dft_along_axis(d, n, ax, re, im, +1);
    memcpy(x, re, sizeof(double) * N);
    free(re); free(im);
}

/*
 * 5th-order WENO reconstruction (Jiang and Shu, 1996) of the numerical flux at
 * the face between v[2] and v[3] from the upwind-biased values v[0..4]
 * (v[0] = f_{i-2} ... v[4] = f_{i+2}): three 3-point candidate fluxes, their
 * smoothness indicators, nonlinear weights from the linear weights
 * (1/10, 6/10, 3/10) with epsilon = 1e-6.
 */
double orc_weno5_face(const double *v)
{
    double q0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    double q1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    double q2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    double b0 = 13.0 / 12.0 * (v[0] - 2.0 * v[1] + v[2]) * (v[0] - 2.0 * v[1] + v[2])
              + 0.25 * (v[0] - 4.0 * v[1] + 3.0 * v[2]) * (v[0] - 4.0 * v[1] + 3.0 * v[2]);
    double b1 = 13.0 / 12.0 * (v[1] - 2.0 * v[2] + v[3]) * (v[1] - 2.0 * v[2] + v[3])
              + 0.25 * (v[1] - v[3]) * (v[1] - v[3]);
    double b2 = 13.0 / 12.0 * (v[2] - 2.0 * v[3] + v[4]) * (v[2] - 2.0 * v[3] + v[4])
              + 0.25 * (3.0 * v[2] - 4.0 * v[3] + v[4]) * (3.0 * v[2] - 4.0 * v[3] + v[4]);
    const double eps = 1e-6;
    double a0 = 0.1 / ((eps + b0) * (eps + b0));
    double a1 = 0.6 / ((eps + b1) * (eps + b1));
    double a2 = 0.3 / ((eps + b2) * (eps + b2));
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/*
 * Advection term of the viscous Burgers equation, f^E(u) = -sum_axes d/dx (u^2/2),
 * by conservative finite differences: F_{i+1/2} = F^+ + F^- with the local
 * Lax-Friedrichs splitting f^(+/-) = (u^2/2 +/- alpha u)/2, alpha = max |u| over the
 * six points i-2..i+3 of the face's stencil; F^+ from f^+_{i-2..i+2}, F^- from
 * f^-_{i+3..i-1} (mirrored); f^E_i -= (F_{i+1/2} - F_{i-1/2}) / h per axis.
 */
static double weno_face_flux(const double *u, int d, int n, int i, int j, int k, int axis)
{
    double w[6], fp[5], fm[5], alpha = 0.0;
    for (int t = 0; t < 6; ++t) {
        int o = t - 2;
        w[t] = u[pidx(d, n, i + (axis == 0) * o, j + (axis == 1) * o, k + (axis == 2) * o)];
        if (fabs(w[t]) > alpha) alpha = fabs(w[t]);
    }
    for (int t = 0; t < 5; ++t) {
        fp[t] = 0.5 * (0.5 * w[t] * w[t] + alpha * w[t]);          /* points i-2..i+2 */
        fm[t] = 0.5 * (0.5 * w[5 - t] * w[5 - t] - alpha * w[5 - t]); /* points i+3..i-1 */
    }
    return orc_weno5_face(fp) + orc_weno5_face(fm);
}

void orc_burgers_advection(int d, int n, const double *u, double *fe)
{
    double h = 2.0 / n;
    for (int k = 0; k < pkmax(d, n); ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int ax = 0; ax < d; ++ax) {
                    double Fr = weno_face_flux(u, d, n, i, j, k, ax);
                    double Fl = weno_face_flux(u, d, n, i - (ax == 0), j - (ax == 1), k - (ax == 2), ax);
                    acc -= (Fr - Fl) / h;
                }
                fe[pidx(d, n, i, j, k)] = acc;
            }
}

/* Multigrid hierarchy: level 0 is the fine grid, sides n_l = (n_{l-1}-1)/2 down to 3. */
typedef struct {
    int d, levels;
    int side[32];
    double *x[32], *b[32], *r[32], *tmp[32];
} orc_mg;

/* Dirichlet: sides n, (n-1)/2, ... down to 3; periodic: n, n/2, ... down to 4. */
static void mg_alloc(orc_mg *mg, int d, int n, int periodic)
{
    memset(mg, 0, sizeof(*mg));
    mg->d = d;
    int s = n, l = 0;
    for (;;) {
        mg->side[l] = s;
        long N = npoints(d, s);
        mg->x[l] = (double *)calloc(N, sizeof(double));
        mg->b[l] = (double *)calloc(N, sizeof(double));
        mg->r[l] = (double *)calloc(N, sizeof(double));
        mg->tmp[l] = (double *)calloc(N, sizeof(double));
        ++l;
        if (periodic ? s <= 4 : s <= 3) break;
        s = periodic ? s / 2 : (s - 1) / 2;
    }
    mg->levels = l;
}

static void mg_free(orc_mg *mg)
{
    for (int l = 0; l < mg->levels; ++l) {
        free(mg->x[l]); free(mg->b[l]); free(mg->r[l]); free(mg->tmp[l]);
    }
}

static void smooth(const orc_problem *P, int n, double a, double *x, const double *b, double *tmp)
{
    if (P->equation == 1) {
        if (P->smoother == 0) orc_smooth_jacobi_per(P->ndim, n, a, P->omega, x, b, tmp);
        else orc_smooth_rbgs_per(P->ndim, n, a, x, b);
    } else if (P->stencil == 1) orc_smooth_jacobi9(n, a, P->omega, x, b, tmp);
    else if (P->smoother == 0) orc_smooth_jacobi(P->ndim, n, a, P->omega, x, b, tmp);
    else orc_smooth_rbgs(P->ndim, n, a, x, b);
}

/* r = b - H x for the problem's operator (I - a L_h, or W - a L_9) */
static void node_residual(const orc_problem *P, int n, double a, const double *x, const double *b, double *r)
{
    if (P->equation == 1) orc_residual_per(P->ndim, n, a, x, b, r);
    else if (P->stencil == 1) orc_residual9(n, a, x, b, r);
    else orc_residual(P->ndim, n, a, x, b, r);
}

/* One V-cycle on level l for H x = b (H = I - a L_{h_l}, or W - a L_9 rediscretised
 * on level l), x updated in place. */
static void vcycle(const orc_problem *P, orc_mg *mg, int l, double a, double *x, const double *b)
{
    int d = P->ndim, n = mg->side[l];
    if (l == mg->levels - 1) { /* coarsest grid: exact solve */
        dense_solve(P->equation == 1 ? 2 : P->stencil, d, n, a, b, x);
        return;
    }
    for (int s = 0; s < P->nu1; ++s) smooth(P, n, a, x, b, mg->tmp[l]);
    node_residual(P, n, a, x, b, mg->r[l]);
    if (P->equation == 1) orc_restrict_per(d, n, mg->r[l], mg->b[l + 1]);
    else orc_restrict_fw(d, n, mg->r[l], mg->b[l + 1]);
    memset(mg->x[l + 1], 0, sizeof(double) * npoints(d, mg->side[l + 1]));
    vcycle(P, mg, l + 1, a, mg->x[l + 1], mg->b[l + 1]);
    if (P->equation == 1) orc_prolong_per(d, mg->side[l + 1], mg->x[l + 1], x);
    else orc_prolong_add(d, mg->side[l + 1], mg->x[l + 1], x);
    for (int s = 0; s < P->nu2; ++s) smooth(P, n, a, x, b, mg->tmp[l]);
}

/* Public single V-cycle (for multigrid tests). */
int orc_vcycle(const orc_problem *P, double a, double *x, const double *b)
{
    orc_mg mg;
    mg_alloc(&mg, P->ndim, P->n, P->equation == 1);
    vcycle(P, &mg, 0, a, x, b);
    mg_free(&mg);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact solve by sine-transform diagonalisation.                           */
/* ------------------------------------------------------------------------ */

/* Apply T[p][i] = sin(i p pi / (n+1)) along one axis (stride 'st'). */
static void sine_along_axis(int d, int n, int axis, double *u, const double *T)
{
    long N = npoints(d, n);
    long st = 1;
    for (int a = 0; a < axis; ++a) st *= n;
#pragma omp parallel
    {
        double *line = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(static)
        for (long base = 0; base < N; ++base) {
            if ((base / st) % n != 0) continue; /* first point of each line */
            for (int p = 0; p < n; ++p) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += T[p * n + i] * u[base + i * st];
                line[p] = acc;
            }
            for (int p = 0; p < n; ++p) u[base + p * st] = line[p];
        }
        free(line);
    }
}

/*
 * Exact solve of (I - a L_h) x = b.  The sine modes
 * v_p(i) = prod_axes sin(i p pi/(n+1)) are eigenvectors of L_h with eigenvalues
 * lambda_p = -(4/h^2) sum_axes sin^2(p pi h / 2); the 1D sine matrix T
 * satisfies T T = (n+1)/2 I.  So x = (2/(n+1))^d T^d diag(1/(1 - a lambda)) T^d b.
 */
void orc_solve_exact(int d, int n, double a, const double *b, double *x)
{
    long N = npoints(d, n);
    double h = 1.0 / (n + 1);
    double *T = (double *)malloc(sizeof(double) * n * n);
    for (int p = 1; p <= n; ++p)
        for (int i = 1; i <= n; ++i)
            T[(p - 1) * n + (i - 1)] = sin(M_PI * (double)i * (double)p / (n + 1));
    memcpy(x, b, sizeof(double) * N);
    for (int ax = 0; ax < d; ++ax) sine_along_axis(d, n, ax, x, T);
    double *lam1 = (double *)malloc(sizeof(double) * n);
    for (int p = 1; p <= n; ++p) {
        double s = sin(M_PI * p * h / 2.0);
        lam1[p - 1] = -4.0 * s * s / (h * h);
    }
    double scale = pow(2.0 / (n + 1), d);
    const int km = kmax(d, n);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k <= km; ++k)
        for (int j = 1; j <= n; ++j)
            for (int i = 1; i <= n; ++i) {
                double lam = lam1[i - 1] + lam1[j - 1] + (d == 3 ? lam1[k - 1] : 0.0);
                x[idx(d, n, i, j, k)] *= scale / (1.0 - a * lam);
            }
    for (int ax = 0; ax < d; ++ax) sine_along_axis(d, n, ax, x, T);
    free(T); free(lam1);
}

/*
 * Exact solve of (W - a L_9) x = b (2D) by the same sine transform: the sine
 * modes are eigenvectors of W and L_9 with eigenvalues
 *   lambda_W = 2/3 + (c_p + c_q)/6,
 *   lambda_9 = (8 (c_p + c_q) + 4 c_p c_q - 20) / (6 h^2),   c_p = cos(p pi h).
 * With a = 0 this applies W^{-1}.
 */
void orc_solve_exact9(int n, double a, const double *b, double *x)
{
    long N = npoints(2, n);
    double h = 1.0 / (n + 1);
    double *T = (double *)calloc((size_t)n * n, sizeof(double));
    for (int p = 1; p <= n; ++p)
        for (int i = 1; i <= n; ++i)
            T[(p - 1) * n + (i - 1)] = sin(M_PI * (double)i * (double)p / (n + 1));
    memcpy(x, b, sizeof(double) * N);
    for (int ax = 0; ax < 2; ++ax) sine_along_axis(2, n, ax, x, T);
    double scale = (2.0 / (n + 1)) * (2.0 / (n + 1));
    for (int j = 1; j <= n; ++j)
        for (int i = 1; i <= n; ++i) {
            double cp = cos(M_PI * i * h), cq = cos(M_PI * j * h);
            double lw = 2.0 / 3.0 + (cp + cq) / 6.0;
            double l9 = (8.0 * (cp + cq) + 4.0 * cp * cq - 20.0) / (6.0 * h * h);
            x[idx(2, n, i, j, 1)] *= scale / (lw - a * l9);
        }
    for (int ax = 0; ax < 2; ++ax) sine_along_axis(2, n, ax, x, T);
    free(T);
}

/* ------------------------------------------------------------------------ */
/* Right-hand side f = f^E + f^I of the ODE system (Sec. 2, Sec. 3).         */
/* ------------------------------------------------------------------------ */
static double f_explicit(const orc_problem *P, double u)
{
    if (P->reaction == 1) return u - u * u * u;
    if (P->reaction == 2) return P->lambda_e * u;
    return 0.0;
}

/* fE = f^E(u) pointwise, fI = nu L_h u (compact stencil: f~^I = W f^I = nu L_9 u) */
static void eval_f(const orc_problem *P, const double *u, double *fE, double *fI)
{
    long N = npoints(P->ndim, P->n);
    if (P->equation == 1) {  /* Burgers: f^I = nu L_h u (periodic), f^E = WENO5 advection */
        orc_laplacian_per(P->ndim, P->n, u, fI);
        orc_burgers_advection(P->ndim, P->n, u, fE);
        for (long p = 0; p < N; ++p) fI[p] *= P->nu;
        return;
    }
    if (P->stencil == 1) orc_laplacian9(P->n, u, fI);
    else orc_laplacian(P->ndim, P->n, u, fI);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        fI[p] *= P->nu;
        fE[p] = f_explicit(P, u[p]);
    }
}

/* ------------------------------------------------------------------------ */
/* One ISDC / SDC time step.                                                 */
/* ------------------------------------------------------------------------ */

/*
 * Advance u (N values, in place) by one time step of length dt.
 *
 * The sweep runs over the points t_0 = T_n and the nodes t_1..t_M of Sec. 2.
 * Gauss-Lobatto has tau_1 = 0, so t_0 is node 1 and a sweep makes M-1 node
 * solves; Gauss-Radau and Gauss-Legendre start at t_0 < t_1 and make M.
 * With Gauss-Legendre (tau_M < 1) the step ends with the collocation
 * end-point quadrature u_{n+1} = u_0 + dt sum_j w_j f(u_j); otherwise
 * u_{n+1} is the last node value.
 *
 * n_sweeps > 0: exactly that many sweeps; n_sweeps == 0: sweep until the SDC
 * residual drops below tol, at most max_sweeps.  n_vcycles is L for solver 0.
 * Outputs: *sweeps_out, *vcycles_out (V-cycles spent on node solves),
 * res_hist[k-1] = residual after sweep k (room for max(n_sweeps, max_sweeps)),
 * nodes_out (optional, M*N): the node values U_1..U_M after the last sweep.
 * nodes_in (optional, M*N): initial node values instead of spreading u (for
 * Gauss-Lobatto its first node must equal u).
 * Returns 0 on success (converged or fixed count), 1 when the cap is hit
 * without convergence, 2 on a non-finite residual, 3 on a bad argument.
 */
int orc_isdc_step(const orc_problem *P, double *u, int n_sweeps, int n_vcycles,
                  int *sweeps_out, long *vcycles_out, double *res_hist, double *nodes_out,
                  const double *nodes_in)
{
    const int d = P->ndim, n = P->n, M = P->M;
    if ((d != 2 && d != 3) || n < 1 || M < 2 || M > ORC_MAX_M) return 3;
    if (P->nodes < 0 || P->nodes > 2) return 3;
    if (P->stencil == 1 && (d != 2 || P->smoother != 0)) return 3; /* compact: 2D, Jacobi */
    if (P->equation == 1 && (P->stencil != 0 || n < 8 || (n & (n - 1)) != 0)) return 3; /* periodic n = 2^j */
    const long N = npoints(d, n);
    const int W9 = P->stencil == 1;
    /* points: t_0 and the nodes; node j (0-based) is point j + off */
    const int off = P->nodes == 0 ? 0 : 1, NP = M + off;
    double tau[ORC_MAX_M], Q[ORC_MAX_M * ORC_MAX_M], w[ORC_MAX_M];
    double tpt[ORC_MAX_M + 1], Qpt[(ORC_MAX_M + 1) * ORC_MAX_M], Spt[ORC_MAX_M * ORC_MAX_M];
    if (orc_nodes(P->nodes, M, tau) != 0) return 3;
    orc_q_matrix(M, tau, Q);
    orc_end_weights(M, tau, w);
    /* Qpt[p][j] = int_0^{t_p} l_j: zero for t_0, the rows of Q for the nodes */
    tpt[0] = 0.0;
    for (int j = 0; j < M; ++j) Qpt[j] = 0.0;
    for (int m = 0; m < M; ++m) {
        tpt[m + off] = tau[m];
        for (int j = 0; j < M; ++j) Qpt[(m + off) * M + j] = Q[m * M + j];
    }
    /* point-to-point integrals S_m^{m+1} = Qpt_{m+1} - Qpt_m (Eq. 2) */
    for (int m = 0; m < NP - 1; ++m)
        for (int j = 0; j < M; ++j) Spt[m * M + j] = Qpt[(m + 1) * M + j] - Qpt[m * M + j];

    /* values at the NP points, old iterate, f^E and f^I */
    double *U = (double *)malloc(sizeof(double) * NP * N);
    double *Uold = (double *)malloc(sizeof(double) * NP * N);
    double *FE = (double *)malloc(sizeof(double) * NP * N);
    double *FI = (double *)malloc(sizeof(double) * NP * N);
    double *FEold = (double *)malloc(sizeof(double) * NP * N);
    double *FIold = (double *)malloc(sizeof(double) * NP * N);
    double *u0 = (double *)malloc(sizeof(double) * N);
    double *rhs = (double *)malloc(sizeof(double) * N);
    double *x = (double *)malloc(sizeof(double) * N);
    double *res = (double *)malloc(sizeof(double) * N);
    double *fe_new = (double *)malloc(sizeof(double) * N);
    double *tmp = (double *)malloc(sizeof(double) * N);
    double *v = (double *)malloc(sizeof(double) * N);
    double *wv = (double *)malloc(sizeof(double) * N);
    orc_mg mg;
    mg_alloc(&mg, d, n, P->equation == 1);

    /* Initial iterate: u_0 spread to every node (the paper does not state it). */
    memcpy(u0, u, sizeof(double) * N);
    memcpy(U, u0, sizeof(double) * N); /* point t_0 */
    for (int m = 0; m < M; ++m)
        if (m + off > 0) memcpy(U + (m + off) * N, nodes_in ? nodes_in + m * N : u0, sizeof(double) * N);
    for (int p = 0; p < NP; ++p) eval_f(P, U + p * N, FE + p * N, FI + p * N);

    int k = 0, status = 0;
    long vcycles = 0;
    int cap = n_sweeps > 0 ? n_sweeps : P->max_sweeps;
    for (;;) {
        /* keep u^k and F(u^k) for the whole sweep */
        copy_values(Uold, U, NP * N);
        copy_values(FEold, FE, NP * N);
        copy_values(FIold, FI, NP * N);

        /* point 0 is t_0: u_0^{k+1} = u_0, nothing to solve */
        for (int m = 0; m < NP - 1; ++m) {
            double dtm = P->dt * (tpt[m + 1] - tpt[m]);
            double a = dtm * P->nu; /* (I - dt_m A) with A = nu L_h */
            const double *Um_new = U + m * N;
            if (P->equation == 1) orc_burgers_advection(d, n, Um_new, fe_new);
            else {
#pragma omp parallel for schedule(static)
                for (long p = 0; p < N; ++p) fe_new[p] = f_explicit(P, Um_new[p]);
            }
            /* Eq. 4 with the implicit unknown moved left:
             * (I - dt_m A) u_{m+1}^{k+1} = u_m^{k+1}
             *     + dt_m [f^E(u_m^{k+1}) - f^E(u_m^k)] - dt_m f^I(u_{m+1}^k)
             *     + S_m^{m+1} F(u^k),   S_m^{m+1}F = dt sum_j s_{m,j} f(u_j^k)
             * (the sum runs over the nodes j, which are points j + off) */
            if (!W9) {
#pragma omp parallel for schedule(static)
                for (long p = 0; p < N; ++p) {
                    double sf = 0.0;
                    for (int j = 0; j < M; ++j)
                        sf += Spt[m * M + j] * (FEold[(j + off) * N + p] + FIold[(j + off) * N + p]);
                    rhs[p] = Um_new[p] + dtm * (fe_new[p] - FEold[m * N + p])
                           - dtm * FIold[(m + 1) * N + p] + P->dt * sf;
                }
            } else {
                /* Eq. 5: W [u_m^{k+1} + dt_m (f^E(u_m^{k+1}) - f^E(u_m^k))] - dt_m A u_{m+1}^k
                 *        + dt sum_j s_{m,j} (W f^E(u_j^k) + A u_j^k),   A u = nu L_9 u = FI */
                for (long p = 0; p < N; ++p) {
                    double se = 0.0;
                    for (int j = 0; j < M; ++j) se += Spt[m * M + j] * FEold[(j + off) * N + p];
                    v[p] = Um_new[p] + dtm * (fe_new[p] - FEold[m * N + p]) + P->dt * se;
                }
                orc_apply_w(n, v, wv);
                for (long p = 0; p < N; ++p) {
                    double si = 0.0;
                    for (int j = 0; j < M; ++j) si += Spt[m * M + j] * FIold[(j + off) * N + p];
                    rhs[p] = wv[p] - dtm * FIold[(m + 1) * N + p] + P->dt * si;
                }
            }
            /* initial guess for the spatial solver (Sec. 4.3) */
            if (P->guess == 0) copy_values(x, Uold + (m + 1) * N, N);
            else if (P->guess == 1) memset(x, 0, sizeof(double) * N);
            else memcpy(x, Um_new, sizeof(double) * N);

            if (P->solver == 2) {
                if (W9) orc_solve_exact9(n, a, rhs, x);
                else if (P->equation == 1) orc_solve_exact_per(d, n, a, rhs, x);
                else orc_solve_exact(d, n, a, rhs, x);
            } else if (P->solver == 1) {
                for (int c = 0; c < P->mg_max_cycles; ++c) {
                    node_residual(P, n, a, x, rhs, tmp);
                    if (max_abs(tmp, N) <= P->mg_tol) break;
                    vcycle(P, &mg, 0, a, x, rhs);
                    ++vcycles;
                }
            } else if (P->solver == 3) {
                for (int c = 0; c < n_vcycles; ++c) {
                    node_residual(P, n, a, x, rhs, tmp);
                    if (max_abs(tmp, N) <= P->mg_tol) break;
                    vcycle(P, &mg, 0, a, x, rhs);
                    ++vcycles;
                }
            } else {
                for (int c = 0; c < n_vcycles; ++c) {
                    vcycle(P, &mg, 0, a, x, rhs);
                    ++vcycles;
                }
            }
            copy_values(U + (m + 1) * N, x, N);
        }
        ++k;

        /* F(u^{k+1}) and the SDC residual
         * max_m max_x | u_0 + dt sum_j q_{m,j} f(u_j^{k+1}) - u_m^{k+1} |   (Sec. 3) */
        for (int p = 0; p < NP; ++p) eval_f(P, U + p * N, FE + p * N, FI + p * N);
        double R = 0.0;
        for (int m = 0; m < M; ++m) {
            if (!W9) {
#pragma omp parallel
                {
                    double Rt = 0.0;
#pragma omp for schedule(static) nowait
                    for (long p = 0; p < N; ++p) {
                        double qf = 0.0;
                        for (int j = 0; j < M; ++j)
                            qf += Q[m * M + j] * (FE[(j + off) * N + p] + FI[(j + off) * N + p]);
                        double r = fabs(u0[p] + P->dt * qf - U[(m + off) * N + p]);
                        if (r > Rt || r != r) Rt = r;
                    }
#pragma omp critical
                    if (Rt > R || Rt != Rt) R = Rt;
                }
            } else {
                /* W r_m = W (u_0 - u_m + dt sum_j q_{m,j} f^E_j) + dt sum_j q_{m,j} A u_j:
                 * one inversion of W per node (Sec. 3) */
                for (long p = 0; p < N; ++p) {
                    double qe = 0.0;
                    for (int j = 0; j < M; ++j) qe += Q[m * M + j] * FE[(j + off) * N + p];
                    v[p] = u0[p] - U[(m + off) * N + p] + P->dt * qe;
                }
                orc_apply_w(n, v, wv);
                for (long p = 0; p < N; ++p) {
                    double qi = 0.0;
                    for (int j = 0; j < M; ++j) qi += Q[m * M + j] * FI[(j + off) * N + p];
                    wv[p] += P->dt * qi;
                }
                orc_solve_exact9(n, 0.0, wv, res);
                for (long p = 0; p < N; ++p) {
                    double r = fabs(res[p]);
                    if (r > R || r != r) R = r;
                }
            }
        }
        if (res_hist) res_hist[k - 1] = R;
        if (!(R == R) || isinf(R)) { status = 2; break; }
        if (n_sweeps > 0) {
            if (k >= n_sweeps) break;
        } else {
            if (R < P->tol) break;
            if (k >= cap) { status = 1; break; }
        }
    }

    if (P->nodes == 2 && !W9) {
        /* Gauss-Legendre: tau_M < 1, end-point quadrature of the collocation rule */
        for (long p = 0; p < N; ++p) {
            double wf = 0.0;
            for (int j = 0; j < M; ++j) wf += w[j] * (FE[(j + off) * N + p] + FI[(j + off) * N + p]);
            u[p] = u0[p] + P->dt * wf;
        }
    } else if (P->nodes == 2) {
        /* the same with f = f^E + W^{-1} A u */
        for (long p = 0; p < N; ++p) {
            double wi = 0.0;
            for (int j = 0; j < M; ++j) wi += w[j] * FI[(j + off) * N + p];
            v[p] = wi;
        }
        orc_solve_exact9(n, 0.0, v, wv);
        for (long p = 0; p < N; ++p) {
            double we = 0.0;
            for (int j = 0; j < M; ++j) we += w[j] * FE[(j + off) * N + p];
            u[p] = u0[p] + P->dt * (we + wv[p]);
        }
    } else {
        memcpy(u, U + (NP - 1) * N, sizeof(double) * N); /* tau_M = 1 */
    }
    if (nodes_out) memcpy(nodes_out, U + off * N, sizeof(double) * M * N);
    if (sweeps_out) *sweeps_out = k;
    if (vcycles_out) *vcycles_out = vcycles;
    free(U); free(Uold); free(FE); free(FI); free(FEold); free(FIold);
    free(u0); free(rhs); free(x); free(res); free(fe_new); free(tmp); free(v); free(wv);
    mg_free(&mg);
    return status;
}

/*
 * SDC residual of given node values (Sec. 3): with f_j = f(U_j),
 *   R = max_m max_x | u_0 + dt sum_j q_{m,j} f_j - U_m |.
 * U: M*N node values.  u0: the step's initial value, or NULL for
 * Gauss-Lobatto (u_0 = U_1).  Used to check a result at sizes where running
 * the whole step on the CPU is too slow.
 */
double orc_sdc_residual(const orc_problem *P, const double *u0, const double *U)
{
    const int M = P->M;
    const long N = npoints(P->ndim, P->n);
    double tau[ORC_MAX_M], Q[ORC_MAX_M * ORC_MAX_M];
    if (orc_nodes(P->nodes, M, tau) != 0 || (!u0 && P->nodes != 0)) return -1.0;
    if (!u0) u0 = U;
    orc_q_matrix(M, tau, Q);
    double *FE = (double *)malloc(sizeof(double) * M * N);
    double *FI = (double *)malloc(sizeof(double) * M * N);
    double *v = (double *)malloc(sizeof(double) * N);
    double *wv = (double *)malloc(sizeof(double) * N);
    double *r9 = (double *)malloc(sizeof(double) * N);
    for (int m = 0; m < M; ++m) eval_f(P, U + m * N, FE + m * N, FI + m * N);
    double R = 0.0;
    for (int m = 0; m < M; ++m) {
        if (P->stencil != 1) {
#pragma omp parallel
            {
                double Rt = 0.0;
#pragma omp for schedule(static) nowait
                for (long p = 0; p < N; ++p) {
                    double qf = 0.0;
                    for (int j = 0; j < M; ++j) qf += Q[m * M + j] * (FE[j * N + p] + FI[j * N + p]);
                    double r = fabs(u0[p] + P->dt * qf - U[m * N + p]);
                    if (r > Rt || r != r) Rt = r;
                }
#pragma omp critical
                if (Rt > R || Rt != Rt) R = Rt;
            }
        } else { /* compact stencil: r_m = W^{-1} [W (u_0 - u_m + dt Q f^E) + dt Q A u] */
            for (long p = 0; p < N; ++p) {
                double qe = 0.0;
                for (int j = 0; j < M; ++j) qe += Q[m * M + j] * FE[j * N + p];
                v[p] = u0[p] - U[m * N + p] + P->dt * qe;
            }
            orc_apply_w(P->n, v, wv);
            for (long p = 0; p < N; ++p) {
                double qi = 0.0;
                for (int j = 0; j < M; ++j) qi += Q[m * M + j] * FI[j * N + p];
                wv[p] += P->dt * qi;
            }
            orc_solve_exact9(P->n, 0.0, wv, r9);
            for (long p = 0; p < N; ++p) {
                double r = fabs(r9[p]);
                if (r > R || r != r) R = r;
            }
        }
    }
    free(FE); free(FI); free(v); free(wv); free(r9);
    return R;
}
