"""ctypes wrapper around ``isdc_oracle.c`` (plain FP64 C, built with gcc).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run this module.

Every function here only marshals arguments; the arithmetic is in the C file,
which follows the paper step by step (Sec. 2 Eq. 2 and Eq. 4, Sec. 3, Sec. 4.3).
Arrays are float64, interior points only, x fastest (C order with shape
(n, n) or (n, n, n) indexed [k, j, i]).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isdc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libisdc_oracle.so")
_OMP_PATH = os.path.join(_BUILD, "libisdc_oracle_omp.so")
_libs = {}
_all_cores = False

SMOOTHER_JACOBI = 0
SMOOTHER_RBGS = 1
SOLVER_ISDC = 0       # L fixed V-cycles per node solve
SOLVER_MG_TOL = 1     # classical SDC: V-cycles until the node residual < mg_tol
SOLVER_EXACT = 2      # classical SDC: exact sine-transform solve
SOLVER_ISDC_CAPPED = 3  # ISDC with L as a cap: stop a node solve early at mg_tol
GUESS_PREVIOUS_SWEEP = 0  # u_{m+1}^k, the paper's choice (Sec. 4.3)
GUESS_ZERO = 1
GUESS_LEFT_NODE = 2       # u_m^{k+1}
REACTION_NONE = 0
REACTION_ALLEN_CAHN = 1   # f^E(u) = u - u^3
REACTION_LINEAR = 2       # f^E(u) = lambda_e * u
NODES_LOBATTO = 0         # Gauss-Lobatto, tau_1 = 0, tau_M = 1 (M - 1 solves per sweep)
NODES_RADAU_RIGHT = 1     # Gauss-Radau, tau_M = 1 (M solves per sweep)
NODES_LEGENDRE = 2        # Gauss-Legendre, interior nodes (M solves, end-point quadrature)
STENCIL_SECOND_ORDER = 0  # 5-point (2D) / 7-point (3D) Laplacian, W = I
STENCIL_COMPACT = 1       # 4th-order compact 9-point Laplacian with weighting matrix W (2D, Sec. 3 Eq. 5)
EQUATION_REACTION_DIFFUSION = 0  # unit square / cube, zero Dirichlet values, n = 2^j - 1 interior points
EQUATION_BURGERS = 1             # viscous Burgers, periodic [-1,1)^d, n = 2^j points, WENO5 advection (Sec. 4.1)


def build(force: bool = False, all_cores: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) if needed: the plain
    build, or (all_cores) the same file with -fopenmp, whose pragmas split the
    outermost grid loops over the host's cores (the same results bit for bit)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _OMP_PATH if all_cores else _LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-D_DEFAULT_SOURCE"] + (["-fopenmp"] if all_cores else ["-Wno-unknown-pragmas"])
                              + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def set_all_cores(enabled: bool) -> None:
    """Route every later call to the OpenMP build (all host cores; OMP_NUM_THREADS
    bounds it) or back to the plain single-threaded build."""
    global _all_cores
    _all_cores = bool(enabled)


class all_cores:
    """Context manager: the oracle runs on all host cores inside the block."""

    def __enter__(self):
        self._prev = _all_cores
        set_all_cores(True)
        return self

    def __exit__(self, *exc):
        set_all_cores(self._prev)
        return False


def threads() -> int:
    """Threads the active build's loops use (1 for the plain build)."""
    return int(_L().orc_threads())


def set_threads(t: int) -> None:
    """Threads for the all-core build's loops (default: OMP_NUM_THREADS or all cores)."""
    with all_cores():
        _L().orc_set_threads(int(t))


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int), ("nu", ctypes.c_double),
                ("M", ctypes.c_int), ("dt", ctypes.c_double), ("reaction", ctypes.c_int),
                ("lambda_e", ctypes.c_double), ("smoother", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("solver", ctypes.c_int), ("guess", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int), ("mg_tol", ctypes.c_double),
                ("mg_max_cycles", ctypes.c_int), ("nodes", ctypes.c_int), ("stencil", ctypes.c_int),
                ("equation", ctypes.c_int)]


@dataclass
class Problem:
    """One ISDC problem (mirrors the C struct ``orc_problem``)."""
    ndim: int
    n: int
    nu: float
    M: int
    dt: float
    reaction: int = REACTION_ALLEN_CAHN
    lambda_e: float = 0.0
    smoother: int = SMOOTHER_JACOBI
    nu1: int = 1
    nu2: int = 1
    omega: float = 2.0 / 3.0
    solver: int = SOLVER_ISDC
    guess: int = GUESS_PREVIOUS_SWEEP
    tol: float = 1e-10
    max_sweeps: int = 50
    mg_tol: float = 1e-12
    mg_max_cycles: int = 100
    nodes: int = NODES_LOBATTO
    stencil: int = STENCIL_SECOND_ORDER
    equation: int = EQUATION_REACTION_DIFFUSION

    def _c(self) -> _Problem:
        return _Problem(self.ndim, self.n, self.nu, self.M, self.dt, self.reaction, self.lambda_e,
                        self.smoother, self.nu1, self.nu2, self.omega, self.solver, self.guess,
                        self.tol, self.max_sweeps, self.mg_tol, self.mg_max_cycles, self.nodes, self.stencil,
                        self.equation)

    @property
    def shape(self):
        return (self.n,) * self.ndim

    @property
    def N(self) -> int:
        return self.n ** self.ndim


def _L():
    key = bool(_all_cores)
    if key not in _libs:
        lib = ctypes.CDLL(build(all_cores=key))
        dp = ctypes.POINTER(ctypes.c_double)
        I, D = ctypes.c_int, ctypes.c_double
        lib.orc_lobatto_nodes.argtypes = [I, dp]
        lib.orc_nodes.argtypes = [I, I, dp]
        lib.orc_end_weights.argtypes = [I, dp, dp]
        lib.orc_q_matrix.argtypes = [I, dp, dp]
        lib.orc_s_matrix.argtypes = [I, dp, dp]
        lib.orc_laplacian.argtypes = [I, I, dp, dp]
        lib.orc_residual.argtypes = [I, I, D, dp, dp, dp]
        lib.orc_smooth_jacobi.argtypes = [I, I, D, D, dp, dp, dp]
        lib.orc_smooth_rbgs.argtypes = [I, I, D, dp, dp]
        lib.orc_restrict_fw.argtypes = [I, I, dp, dp]
        lib.orc_prolong_add.argtypes = [I, I, dp, dp]
        lib.orc_dense_solve.argtypes = [I, I, D, dp, dp]
        lib.orc_solve_exact.argtypes = [I, I, D, dp, dp]
        lib.orc_laplacian9.argtypes = [I, dp, dp]
        lib.orc_apply_w.argtypes = [I, dp, dp]
        lib.orc_residual9.argtypes = [I, D, dp, dp, dp]
        lib.orc_smooth_jacobi9.argtypes = [I, D, D, dp, dp, dp]
        lib.orc_dense_solve9.argtypes = [I, D, dp, dp]
        lib.orc_solve_exact9.argtypes = [I, D, dp, dp]
        lib.orc_laplacian_per.argtypes = [I, I, dp, dp]
        lib.orc_residual_per.argtypes = [I, I, D, dp, dp, dp]
        lib.orc_smooth_jacobi_per.argtypes = [I, I, D, D, dp, dp, dp]
        lib.orc_smooth_rbgs_per.argtypes = [I, I, D, dp, dp]
        lib.orc_restrict_per.argtypes = [I, I, dp, dp]
        lib.orc_prolong_per.argtypes = [I, I, dp, dp]
        lib.orc_solve_exact_per.argtypes = [I, I, D, dp, dp]
        lib.orc_weno5_face.argtypes = [dp]
        lib.orc_weno5_face.restype = D
        lib.orc_burgers_advection.argtypes = [I, I, dp, dp]
        lib.orc_vcycle.argtypes = [ctypes.POINTER(_Problem), D, dp, dp]
        lib.orc_isdc_step.argtypes = [ctypes.POINTER(_Problem), dp, I, I, ctypes.POINTER(I),
                                      ctypes.POINTER(ctypes.c_long), dp, dp, dp]
        lib.orc_sdc_residual.argtypes = [ctypes.POINTER(_Problem), dp, dp]
        lib.orc_sdc_residual.restype = D
        lib.orc_threads.argtypes = []
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = None
        for f in ("orc_lobatto_nodes", "orc_nodes", "orc_end_weights", "orc_q_matrix", "orc_s_matrix",
                  "orc_vcycle", "orc_isdc_step", "orc_threads"):
            getattr(lib, f).restype = I
        _libs[key] = lib
    return _libs[key]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --- quadrature (Sec. 2, Eq. 2) ---------------------------------------------
def lobatto_nodes(M: int) -> np.ndarray:
    tau = np.zeros(M)
    if _L().orc_lobatto_nodes(M, _p(tau)):
        raise ValueError("bad M")
    return tau


def nodes(M: int, kind: int = NODES_LOBATTO) -> np.ndarray:
    """Collocation nodes tau_1 < ... < tau_M on [0, 1] of the given family (Sec. 2)."""
    tau = np.zeros(M)
    if _L().orc_nodes(kind, M, _p(tau)):
        raise ValueError("bad M or node family")
    return tau


def q_matrix(M: int, kind: int = NODES_LOBATTO) -> np.ndarray:
    """Q[m, j] = int_0^{tau_m} l_j (Eq. 2)."""
    tau = nodes(M, kind)
    Q = np.zeros((M, M))
    _L().orc_q_matrix(M, _p(tau), _p(Q))
    return Q


def end_weights(M: int, kind: int = NODES_LOBATTO) -> np.ndarray:
    """w_j = int_0^1 l_j: the collocation rule's weights over the whole step."""
    tau = nodes(M, kind)
    w = np.zeros(M)
    _L().orc_end_weights(M, _p(tau), _p(w))
    return w


def s_matrix(M: int) -> np.ndarray:
    Q = q_matrix(M)
    S = np.zeros((M - 1, M))
    _L().orc_s_matrix(M, _p(Q), _p(S))
    return S


# --- spatial operators and multigrid components ------------------------------
def _dims(u: np.ndarray):
    d = u.ndim
    n = u.shape[0]
    assert all(s == n for s in u.shape)
    return d, n


def laplacian(u):
    u = _f64(u)
    d, n = _dims(u)
    out = np.empty_like(u)
    _L().orc_laplacian(d, n, _p(u), _p(out))
    return out


def residual(a, x, b):
    x, b = _f64(x), _f64(b)
    d, n = _dims(x)
    r = np.empty_like(x)
    _L().orc_residual(d, n, a, _p(x), _p(b), _p(r))
    return r


def smooth_jacobi(a, omega, x, b):
    x, b = _f64(x).copy(), _f64(b)
    d, n = _dims(x)
    tmp = np.empty_like(x)
    _L().orc_smooth_jacobi(d, n, a, omega, _p(x), _p(b), _p(tmp))
    return x


def smooth_rbgs(a, x, b):
    x, b = _f64(x).copy(), _f64(b)
    d, n = _dims(x)
    _L().orc_smooth_rbgs(d, n, a, _p(x), _p(b))
    return x


def restrict_fw(r):
    r = _f64(r)
    d, n = _dims(r)
    nc = (n - 1) // 2
    rc = np.zeros((nc,) * d)
    _L().orc_restrict_fw(d, n, _p(r), _p(rc))
    return rc


def prolong_add(ec, x):
    ec, x = _f64(ec), _f64(x).copy()
    d, nc = _dims(ec)
    assert x.shape[0] == 2 * nc + 1
    _L().orc_prolong_add(d, nc, _p(ec), _p(x))
    return x


def dense_solve(a, b):
    b = _f64(b)
    d, n = _dims(b)
    x = np.zeros_like(b)
    _L().orc_dense_solve(d, n, a, _p(b), _p(x))
    return x


# --- 4th-order compact discretisation (Sec. 3, Eq. 5), 2D ----------------------
def _dims2(u: np.ndarray):
    d, n = _dims(u)
    assert d == 2, "the compact stencil is 2D"
    return n


def laplacian9(u):
    """The 9-point compact Laplacian L_9 u."""
    u = _f64(u)
    n = _dims2(u)
    out = np.empty_like(u)
    _L().orc_laplacian9(n, _p(u), _p(out))
    return out


def apply_w(u):
    """The weighting matrix W u = u + (h^2/12) L_5 u."""
    u = _f64(u)
    n = _dims2(u)
    out = np.empty_like(u)
    _L().orc_apply_w(n, _p(u), _p(out))
    return out


def residual9(a, x, b):
    x, b = _f64(x), _f64(b)
    n = _dims2(x)
    r = np.empty_like(x)
    _L().orc_residual9(n, a, _p(x), _p(b), _p(r))
    return r


def smooth_jacobi9(a, omega, x, b):
    x, b = _f64(x).copy(), _f64(b)
    n = _dims2(x)
    tmp = np.empty_like(x)
    _L().orc_smooth_jacobi9(n, a, omega, _p(x), _p(b), _p(tmp))
    return x


def dense_solve9(a, b):
    b = _f64(b)
    n = _dims2(b)
    x = np.zeros_like(b)
    _L().orc_dense_solve9(n, a, _p(b), _p(x))
    return x


def solve_exact9(a, b):
    """(W - a L_9)^{-1} b by the sine transform (a = 0: W^{-1} b)."""
    b = _f64(b)
    n = _dims2(b)
    x = np.zeros_like(b)
    _L().orc_solve_exact9(n, a, _p(b), _p(x))
    return x


def solve_exact(a, b):
    b = _f64(b)
    d, n = _dims(b)
    x = np.zeros_like(b)
    _L().orc_solve_exact(d, n, a, _p(b), _p(x))
    return x


def vcycle(problem: Problem, a, x, b):
    x, b = _f64(x).copy(), _f64(b)
    pc = problem._c()
    _L().orc_vcycle(ctypes.byref(pc), a, _p(x), _p(b))
    return x


# --- one ISDC / SDC time step (Sec. 2 Eq. 4, Sec. 3) ---------------------------
@dataclass
class StepResult:
    u: np.ndarray
    sweeps: int
    vcycles: int
    residuals: np.ndarray
    status: int
    nodes: np.ndarray | None = None


def isdc_step(problem: Problem, u, n_sweeps: int = 0, n_vcycles: int = 2,
              want_nodes: bool = False, nodes_in=None) -> StepResult:
    """One time step from u (returns u at T_n + dt).  n_sweeps=0: until tol."""
    u = _f64(u).copy()
    assert u.shape == problem.shape
    cap = max(n_sweeps, problem.max_sweeps)
    hist = np.zeros(cap)
    nodes = np.zeros((problem.M,) + problem.shape) if want_nodes else None
    nin = None
    if nodes_in is not None:
        nin = _f64(nodes_in)
        assert nin.shape == (problem.M,) + problem.shape
    sweeps = ctypes.c_int(0)
    vcyc = ctypes.c_long(0)
    pc = problem._c()
    st = _L().orc_isdc_step(ctypes.byref(pc), _p(u), n_sweeps, n_vcycles, ctypes.byref(sweeps),
                            ctypes.byref(vcyc), _p(hist), _p(nodes) if nodes is not None else None,
                            _p(nin) if nin is not None else None)
    if st == 3:
        raise ValueError("invalid problem")
    return StepResult(u, sweeps.value, vcyc.value, hist[:sweeps.value].copy(), st, nodes)


def sdc_residual(problem: Problem, node_values, u0=None) -> float:
    """Max-norm SDC residual (Sec. 3) of node values (shape (M,) + grid); u0 is
    the step's initial value (for Gauss-Lobatto it defaults to the first node)."""
    node_values = _f64(node_values)
    assert node_values.shape == (problem.M,) + problem.shape
    u0p = None
    if u0 is not None:
        u0 = _f64(u0)
        assert u0.shape == problem.shape
        u0p = _p(u0)
    pc = problem._c()
    R = float(_L().orc_sdc_residual(ctypes.byref(pc), u0p, _p(node_values)))
    if R < 0:
        raise ValueError("invalid problem (u0 is required for this node family)")
    return R


@dataclass
class RunResult:
    u: np.ndarray
    per_step_u: list = field(default_factory=list)
    sweeps: list = field(default_factory=list)
    vcycles: list = field(default_factory=list)
    residuals: list = field(default_factory=list)
    status: list = field(default_factory=list)


def integrate(problem: Problem, u0, steps: int, n_sweeps=0, n_vcycles: int = 2,
              keep_steps: bool = True) -> RunResult:
    """Run several time steps; n_sweeps may be an int or a per-step list."""
    u = _f64(u0).copy()
    out = RunResult(u)
    for s in range(steps):
        ns = n_sweeps[s] if isinstance(n_sweeps, (list, tuple, np.ndarray)) else n_sweeps
        r = isdc_step(problem, u, int(ns), n_vcycles)
        u = r.u
        if keep_steps:
            out.per_step_u.append(u.copy())
        out.sweeps.append(r.sweeps)
        out.vcycles.append(r.vcycles)
        out.residuals.append(r.residuals)
        out.status.append(r.status)
    out.u = u
    return out


# --- periodic grids and WENO5 advection (viscous Burgers, Sec. 4.1) ------------
def laplacian_per(u):
    u = _f64(u)
    d, n = _dims(u)
    out = np.empty_like(u)
    _L().orc_laplacian_per(d, n, _p(u), _p(out))
    return out


def residual_per(a, x, b):
    x, b = _f64(x), _f64(b)
    d, n = _dims(x)
    r = np.empty_like(x)
    _L().orc_residual_per(d, n, a, _p(x), _p(b), _p(r))
    return r


def smooth_jacobi_per(a, omega, x, b):
    x, b = _f64(x).copy(), _f64(b)
    d, n = _dims(x)
    tmp = np.empty_like(x)
    _L().orc_smooth_jacobi_per(d, n, a, omega, _p(x), _p(b), _p(tmp))
    return x


def smooth_rbgs_per(a, x, b):
    x, b = _f64(x).copy(), _f64(b)
    d, n = _dims(x)
    _L().orc_smooth_rbgs_per(d, n, a, _p(x), _p(b))
    return x


def restrict_per(r):
    r = _f64(r)
    d, n = _dims(r)
    rc = np.zeros((n // 2,) * d)
    _L().orc_restrict_per(d, n, _p(r), _p(rc))
    return rc


def prolong_per(ec, x):
    ec, x = _f64(ec), _f64(x).copy()
    d, nc = _dims(ec)
    assert x.shape[0] == 2 * nc
    _L().orc_prolong_per(d, nc, _p(ec), _p(x))
    return x


def solve_exact_per(a, b):
    """(I - a L_h)^{-1} b on the periodic grid by the discrete Fourier transform."""
    b = _f64(b)
    d, n = _dims(b)
    x = np.zeros_like(b)
    _L().orc_solve_exact_per(d, n, a, _p(b), _p(x))
    return x


def weno5_face(v):
    """WENO5 face value from the five upwind-biased values v[0..4]."""
    v = _f64(v)
    assert v.shape == (5,)
    return float(_L().orc_weno5_face(_p(v)))


def burgers_advection(u):
    """f^E(u) = -sum_axes (u^2/2)_x by WENO5 with local Lax-Friedrichs splitting (periodic)."""
    u = _f64(u)
    d, n = _dims(u)
    out = np.empty_like(u)
    _L().orc_burgers_advection(d, n, _p(u), _p(out))
    return out
