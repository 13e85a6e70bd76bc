"""Thin ctypes binding of the C ABI in include/isdc.h (libisdc.so).

Every function has the name of the C entry point it calls and only marshals
arguments (torch tensors -> device pointers, options -> the C struct).  All
compute runs in the CUDA kernels of libisdc.so; there is no fallback: if the
library cannot be loaded, or a tensor is not a contiguous float64 CUDA
tensor, the call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

ISDC_OK = 0
ISDC_ERR_INVALID_ARG = 1
ISDC_ERR_UNSUPPORTED = 2
ISDC_ERR_OOM = 3
ISDC_ERR_CUDA = 4
ISDC_ERR_NOT_CONVERGED = 5
ISDC_ERR_NONFINITE = 6
ISDC_ERR_SCRATCH_TOO_SMALL = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "NOT_CONVERGED",
                6: "NONFINITE", 7: "SCRATCH_TOO_SMALL"}
ISDC_STATIC_SCRATCH_BYTES = 64 << 20

ISDC_NODES_GAUSS_LOBATTO = 0
ISDC_NODES_RADAU_RIGHT = 1
ISDC_NODES_GAUSS_LEGENDRE = 2
ISDC_SMOOTHER_JACOBI = 0
ISDC_SMOOTHER_RBGS = 1
ISDC_REACTION_NONE = 0
ISDC_REACTION_ALLEN_CAHN = 1
ISDC_STENCIL_SECOND_ORDER = 0
ISDC_STENCIL_COMPACT = 1
ISDC_EQUATION_REACTION_DIFFUSION = 0
ISDC_EQUATION_BURGERS = 1


class isdc_options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("vcycle_fp32", ctypes.c_int), ("reaction", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int), ("mg_tol", ctypes.c_double),
                ("mg_max_cycles", ctypes.c_int), ("vcycle_cap", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("temporal_blocking", ctypes.c_int), ("stencil", ctypes.c_int),
                ("equation", ctypes.c_int), ("rb_run", ctypes.c_int), ("fused_transfer", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class isdc_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("fp64_ops", ctypes.c_double), ("fp32_ops", ctypes.c_double)]


class isdc_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nu", ctypes.c_double), ("M", ctypes.c_int), ("dt", ctypes.c_double),
                ("steps", ctypes.c_int)]


class isdc_slot_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("steps_done", ctypes.c_int), ("sweeps_in_step", ctypes.c_int),
                ("total_sweeps", ctypes.c_int), ("nonconverged_steps", ctypes.c_int),
                ("last_residual", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


class isdc_batch_info(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("running", ctypes.c_int),
                ("tuned", ctypes.c_int), ("threads_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("fused", ctypes.c_int), ("kernels_per_tick", ctypes.c_int), ("bytes_last_tick", ctypes.c_double),
                ("lanes", ctypes.c_int), ("lane_split", ctypes.c_int)]


ISDC_SLOT_FREE, ISDC_SLOT_RUNNING, ISDC_SLOT_FINISHED, ISDC_SLOT_FAILED = 0, 1, 2, 3


class IsdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_ctx_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB


_probe = None


def probe_fp64_rate():
    """The GPU's FP64 issue rate (FP64 operations per second; one FMA = one
    operation) measured by libisdc_probe.so, and the best launch's ms."""
    global _probe
    if _probe is None:
        path = _build.build_probe()
        if not os.path.exists(path):
            raise RuntimeError(f"probe library {path} is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.isdc_probe_fp64_rate.argtypes = [_dp, _dp]
        lib.isdc_probe_fp64_rate.restype = ctypes.c_int
        _probe = lib
    ops, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = _probe.isdc_probe_fp64_rate(ctypes.byref(ops), ctypes.byref(ms))
    if st != 0:
        raise RuntimeError(f"isdc_probe_fp64_rate failed ({st})")
    return ops.value, ms.value


def load(build_if_missing: bool = True):
    """Load libisdc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    I, D, V = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "isdc_default_options": (I, [ctypes.POINTER(isdc_options)]),
        "isdc_collocation_tables": (I, [I, I, _dp, _dp, _dp]),
        "isdc_create": (I, [I, ctypes.POINTER(ctypes.c_int64), D, I, I, D, ctypes.POINTER(isdc_options),
                            ctypes.POINTER(_ctx_p)]),
        "isdc_step": (I, [_ctx_p, V, I, I]),
        "isdc_step_host": (I, [_ctx_p, V, I, I]),
        "isdc_residual": (I, [_ctx_p, _dp]),
        "isdc_stats": (I, [_ctx_p, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_int64)]),
        "isdc_residual_history": (I, [_ctx_p, _dp, I, ctypes.POINTER(I)]),
        "isdc_set_record_history": (I, [_ctx_p, I]),
        "isdc_get_nodes": (I, [_ctx_p, V]),
        "isdc_set_nodes": (I, [_ctx_p, V]),
        "isdc_vcycles": (I, [_ctx_p, D, V, V, I]),
        "isdc_vcycles_static": (I, [I, ctypes.c_int64, D, I, I, I, D, V, V, I, V]),
        "isdc_batch_create": (I, [I, ctypes.c_int64, I, ctypes.c_size_t, I, ctypes.POINTER(isdc_options),
                                  ctypes.POINTER(_ctx_p)]),
        "isdc_batch_admit": (I, [_ctx_p, ctypes.POINTER(isdc_problem), V, I, ctypes.POINTER(I)]),
        "isdc_batch_tick": (I, [_ctx_p, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "isdc_batch_query": (I, [_ctx_p, I, ctypes.POINTER(isdc_slot_info)]),
        "isdc_batch_take": (I, [_ctx_p, I, V, I]),
        "isdc_batch_stats": (I, [_ctx_p, ctypes.POINTER(isdc_batch_info)]),
        "isdc_batch_last_error": (ctypes.c_char_p, [_ctx_p]),
        "isdc_batch_destroy": (None, [_ctx_p]),
        "isdc_batch_barrier_selftest": (I, [I, I, ctypes.c_double, ctypes.POINTER(I)]),
        "isdc_profile_enable": (I, [_ctx_p, I]),
        "isdc_profile_read": (I, [_ctx_p, ctypes.POINTER(isdc_kernel_stat), I, ctypes.POINTER(I)]),
        "isdc_tuning": (I, [_ctx_p, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "isdc_tuning_transfer": (I, [_ctx_p, ctypes.POINTER(I), I, ctypes.POINTER(I)]),
        "isdc_last_error": (ctypes.c_char_p, [_ctx_p]),
        "isdc_destroy": (None, [_ctx_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st, ctx=None, soft=()):
    if st != ISDC_OK and st not in soft:
        raise IsdcError(st, load().isdc_last_error(ctx).decode(errors="replace"))
    return st


def _dev_ptr(t, numel=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} values, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


# --- C entry points ---------------------------------------------------------
def isdc_default_options() -> isdc_options:
    o = isdc_options()
    _check(load().isdc_default_options(ctypes.byref(o)))
    return o


def isdc_collocation_tables(M: int, nodes: int = ISDC_NODES_GAUSS_LOBATTO):
    """Host-only tables (tau, Q, S) as nested lists; S has one row per sweep
    step between consecutive points (M - 1 for Gauss-Lobatto, else M)."""
    rows = M - 1 if nodes == ISDC_NODES_GAUSS_LOBATTO else M
    tau = (ctypes.c_double * M)()
    Q = (ctypes.c_double * (M * M))()
    S = (ctypes.c_double * (rows * M))()
    _check(load().isdc_collocation_tables(nodes, M, tau, Q, S))
    return (list(tau), [list(Q[m * M:(m + 1) * M]) for m in range(M)],
            [list(S[m * M:(m + 1) * M]) for m in range(rows)])


def isdc_create(ndim, n, nu, M, dt, options: isdc_options | None = None,
                nodes: int = ISDC_NODES_GAUSS_LOBATTO):
    dims = (ctypes.c_int64 * ndim)(*([n] * ndim))
    out = _ctx_p()
    st = load().isdc_create(ndim, dims, nu, nodes, M, dt,
                            ctypes.byref(options) if options is not None else None, ctypes.byref(out))
    _check(st)
    return out


def isdc_step(ctx, u, n_sweeps: int, n_vcycles: int) -> int:
    """u: float64 CUDA tensor (n^ndim values).  Returns OK or NOT_CONVERGED."""
    return _check(load().isdc_step(ctx, _dev_ptr(u), n_sweeps, n_vcycles), ctx, soft=(ISDC_ERR_NOT_CONVERGED,))


def isdc_step_host(ctx, u_host, n_sweeps: int, n_vcycles: int) -> int:
    """u_host: contiguous float64 host buffer (numpy array or CPU tensor)."""
    import numpy as np
    if isinstance(u_host, np.ndarray):
        if u_host.dtype != np.float64 or not u_host.flags.c_contiguous:
            raise TypeError("expected a contiguous float64 array")
        ptr = ctypes.c_void_p(u_host.ctypes.data)
    else:
        import torch
        if u_host.is_cuda or u_host.dtype != torch.float64 or not u_host.is_contiguous():
            raise TypeError("expected a contiguous float64 CPU tensor")
        ptr = ctypes.c_void_p(u_host.data_ptr())
    return _check(load().isdc_step_host(ctx, ptr, n_sweeps, n_vcycles), ctx, soft=(ISDC_ERR_NOT_CONVERGED,))


def isdc_residual(ctx) -> float:
    r = ctypes.c_double()
    _check(load().isdc_residual(ctx, ctypes.byref(r)), ctx)
    return r.value


def isdc_stats(ctx):
    s, v = ctypes.c_int(), ctypes.c_int64()
    _check(load().isdc_stats(ctx, ctypes.byref(s), ctypes.byref(v)), ctx)
    return s.value, v.value


def isdc_residual_history(ctx, cap: int = 100000):
    cnt = ctypes.c_int()
    _check(load().isdc_residual_history(ctx, None, 0, ctypes.byref(cnt)), ctx)
    buf = (ctypes.c_double * max(1, min(cap, cnt.value)))()
    _check(load().isdc_residual_history(ctx, buf, min(cap, cnt.value), ctypes.byref(cnt)), ctx)
    return list(buf[:min(cap, cnt.value)])


def isdc_set_record_history(ctx, record: bool):
    _check(load().isdc_set_record_history(ctx, 1 if record else 0), ctx)


def isdc_get_nodes(ctx, dst):
    _check(load().isdc_get_nodes(ctx, _dev_ptr(dst)), ctx)


def isdc_set_nodes(ctx, src):
    _check(load().isdc_set_nodes(ctx, _dev_ptr(src)), ctx)


def isdc_vcycles(ctx, a: float, x, b, n_cycles: int):
    _check(load().isdc_vcycles(ctx, a, _dev_ptr(x), _dev_ptr(b, x.numel()), n_cycles), ctx)


def isdc_vcycles_static(ndim, n, a: float, x, b, n_cycles: int, smoother=ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1,
                        omega=2.0 / 3.0, stream=None):
    """The allocation-free multigrid solve (no context; scratch in a static
    device array).  Runs on `stream` (a torch CUDA stream; default: torch's
    current stream).  Raises IsdcError with the status on failure."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    h = ctypes.c_void_p(s.cuda_stream if s.cuda_stream else None)
    st = load().isdc_vcycles_static(ndim, n, a, smoother, nu1, nu2, omega, _dev_ptr(x), _dev_ptr(b, x.numel()),
                                    n_cycles, h)
    if st != ISDC_OK:
        raise IsdcError(st, "isdc_vcycles_static failed"
                        + (f" (its scratch holds {ISDC_STATIC_SCRATCH_BYTES} bytes: 2D sides up to 1023, "
                           "3D sides up to 127)" if st == ISDC_ERR_SCRATCH_TOO_SMALL else ""))
    return st


PROFILE_CLASSES = ["spread", "eval_f", "rhs", "sweep_end", "smooth_fine", "residual_fine", "restrict_fine",
                   "prolong_fine", "smooth_coarse", "residual_coarse", "restrict_coarse", "prolong_coarse",
                   "bottom", "defect", "update", "resnorm", "w_inverse", "resrestrict_fine", "resrestrict_coarse"]


def isdc_profile_enable(ctx, enable, classes=None):
    """enable: False = off; True = time every class with events, or only the
    named `classes` (counts, bytes and ops are kept for all; classes=[] counts
    only, with no events and no per-sweep synchronisation)."""
    if not enable:
        mask = 0
    elif classes is None:
        mask = -1
    else:
        mask = 1 << 30 if not classes else 0
        for c in classes:
            mask |= 1 << PROFILE_CLASSES.index(c)
    _check(load().isdc_profile_enable(ctx, mask), ctx)


def isdc_profile_read(ctx):
    """{class name: dict(launches, total_ms, bytes, fp64_ops, fp32_ops)}"""
    cnt = ctypes.c_int()
    buf = (isdc_kernel_stat * 64)()
    _check(load().isdc_profile_read(ctx, buf, 64, ctypes.byref(cnt)), ctx)
    out = {}
    for r in buf[:min(cnt.value, 64)]:
        out[r.name.decode()] = dict(launches=r.launches, total_ms=r.total_ms, bytes=r.bytes,
                                    fp64_ops=r.fp64_ops, fp32_ops=r.fp32_ops)
    return out


def isdc_tuning(ctx):
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().isdc_tuning(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), ctx)
    kc = (ctypes.c_int * 16)()
    nl = ctypes.c_int()
    _check(load().isdc_tuning_transfer(ctx, kc, 16, ctypes.byref(nl)), ctx)
    return {"zb_fp64": a.value, "zb_fp32": b.value, "tb_depth": c.value, "tb_planes": d.value,
            "transfer_kc": [kc[i] for i in range(min(nl.value, 16))]}


def isdc_last_error(ctx=None) -> str:
    return load().isdc_last_error(ctx).decode(errors="replace")


def isdc_destroy(ctx):
    if ctx:
        load().isdc_destroy(ctx)


# --- batched engine -----------------------------------------------------------------
def _bcheck(st, b=None, soft=()):
    if st != ISDC_OK and st not in soft:
        raise IsdcError(st, load().isdc_batch_last_error(b).decode(errors="replace"))
    return st


def isdc_batch_create(ndim, max_side, max_M, hbm_budget_bytes, n_vcycles, options: isdc_options | None = None):
    out = _ctx_p()
    _bcheck(load().isdc_batch_create(ndim, max_side, max_M, hbm_budget_bytes, n_vcycles,
                                     ctypes.byref(options) if options is not None else None, ctypes.byref(out)))
    return out


def isdc_batch_admit(b, n, nu, M, dt, steps, u0):
    """u0: numpy float64 array (host) or float64 CUDA tensor (device).  Returns
    the slot, or None when the budget or the slots are exhausted (soft)."""
    import numpy as np
    p = isdc_problem(n, nu, M, dt, steps)
    if isinstance(u0, np.ndarray):
        if u0.dtype != np.float64 or not u0.flags.c_contiguous:
            raise TypeError("expected a contiguous float64 array")
        ptr, host = ctypes.c_void_p(u0.ctypes.data), 1
    else:
        ptr, host = _dev_ptr(u0), 0
    slot = ctypes.c_int(-1)
    st = _bcheck(load().isdc_batch_admit(b, ctypes.byref(p), ptr, host, ctypes.byref(slot)), b,
                 soft=(ISDC_ERR_OOM,))
    return None if st == ISDC_ERR_OOM else slot.value


def isdc_batch_tick(b):
    r, f = ctypes.c_int(), ctypes.c_int()
    _bcheck(load().isdc_batch_tick(b, ctypes.byref(r), ctypes.byref(f)), b)
    return r.value, f.value


def isdc_batch_query(b, slot):
    info = isdc_slot_info()
    _bcheck(load().isdc_batch_query(b, slot, ctypes.byref(info)), b)
    return info


def isdc_batch_take(b, slot, out=None):
    """Copy the finished solution into `out` (numpy float64 array or float64 CUDA
    tensor; None discards it) and free the slot."""
    import numpy as np
    if out is None:
        ptr, host = None, 0
    elif isinstance(out, np.ndarray):
        ptr, host = ctypes.c_void_p(out.ctypes.data), 1
    else:
        ptr, host = _dev_ptr(out), 0
    _bcheck(load().isdc_batch_take(b, slot, ptr, host), b)


def isdc_batch_stats(b):
    info = isdc_batch_info()
    _bcheck(load().isdc_batch_stats(b, ctypes.byref(info)), b)
    return info


def isdc_batch_destroy(b):
    if b:
        load().isdc_batch_destroy(b)


class Batch:
    """An engine for many independent ISDC integrations of one dimension."""

    def __init__(self, ndim, max_side, max_M=5, hbm_budget_bytes=64 << 30, n_vcycles=2, *,
                 smoother=ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, omega=2.0 / 3.0, reaction=ISDC_REACTION_ALLEN_CAHN,
                 tol=1e-10, max_sweeps=100, temporal_blocking=-1):
        o = isdc_default_options()
        o.smoother, o.nu1, o.nu2, o.omega, o.reaction = smoother, nu1, nu2, omega, reaction
        o.tol, o.max_sweeps, o.vcycle_fp32 = tol, max_sweeps, 1
        o.temporal_blocking = int(temporal_blocking)
        self.ndim = ndim
        self.b = isdc_batch_create(ndim, max_side, max_M, hbm_budget_bytes, n_vcycles, o)
        self.sides = {}

    def admit(self, n, nu, M, dt, steps, u0):
        slot = isdc_batch_admit(self.b, n, nu, M, dt, steps, u0)
        if slot is not None:
            self.sides[slot] = n
        return slot

    def tick(self):
        return isdc_batch_tick(self.b)

    def query(self, slot):
        return isdc_batch_query(self.b, slot)

    def take(self, slot):
        import numpy as np
        out = np.empty((self.sides[slot],) * self.ndim)
        isdc_batch_take(self.b, slot, out)
        del self.sides[slot]
        return out

    def stats(self):
        return isdc_batch_stats(self.b)

    def close(self):
        if self.b:
            isdc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- convenience wrapper ------------------------------------------------------
class Isdc:
    """One ISDC problem on the GPU.  By default it runs on torch's current
    CUDA stream so that torch events and tensors order with it."""

    def __init__(self, ndim, n, nu, M, dt, *, smoother=ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1,
                 omega=2.0 / 3.0, vcycle_fp32=False, reaction=ISDC_REACTION_ALLEN_CAHN, tol=1e-10,
                 max_sweeps=100, mg_tol=1e-12, mg_max_cycles=50, vcycle_cap=False, use_graphs=True,
                 temporal_blocking=-1, nodes=ISDC_NODES_GAUSS_LOBATTO, stencil=ISDC_STENCIL_SECOND_ORDER,
                 equation=ISDC_EQUATION_REACTION_DIFFUSION, rb_run=0, fused_transfer=-1, stream=None):
        import torch
        o = isdc_default_options()
        o.smoother, o.nu1, o.nu2, o.omega = smoother, nu1, nu2, omega
        o.vcycle_fp32, o.reaction, o.tol, o.max_sweeps = int(vcycle_fp32), reaction, tol, max_sweeps
        o.mg_tol, o.mg_max_cycles, o.vcycle_cap = mg_tol, mg_max_cycles, int(vcycle_cap)
        o.use_graphs, o.temporal_blocking, o.stencil = int(use_graphs), int(temporal_blocking), int(stencil)
        o.equation, o.rb_run, o.fused_transfer = int(equation), int(rb_run), int(fused_transfer)
        s = stream if stream is not None else torch.cuda.current_stream()
        # torch's default stream has handle 0, which the C ABI reads as "create a
        # private stream"; pass cudaStreamLegacy (1) so the work orders with torch.
        o.stream = ctypes.c_void_p(s.cuda_stream if s.cuda_stream else 1)
        self.stream = s
        self.ndim, self.n, self.M = ndim, n, M
        self.N = n ** ndim
        self.ctx = isdc_create(ndim, n, nu, M, dt, o, nodes)

    def step(self, u, n_sweeps=0, n_vcycles=2):
        return isdc_step(self.ctx, u, n_sweeps, n_vcycles)

    def step_host(self, u_host, n_sweeps=0, n_vcycles=2):
        return isdc_step_host(self.ctx, u_host, n_sweeps, n_vcycles)

    def residual(self):
        return isdc_residual(self.ctx)

    def stats(self):
        return isdc_stats(self.ctx)

    def history(self):
        return isdc_residual_history(self.ctx)

    def record_history(self, on=True):
        isdc_set_record_history(self.ctx, on)

    def nodes(self):
        import torch
        out = torch.empty((self.M,) + (self.n,) * self.ndim, dtype=torch.float64, device="cuda")
        isdc_get_nodes(self.ctx, out)
        return out

    def set_nodes(self, nodes):
        isdc_set_nodes(self.ctx, nodes.contiguous())

    def vcycles(self, a, x, b, n_cycles):
        isdc_vcycles(self.ctx, a, x, b, n_cycles)

    def tuning(self):
        return isdc_tuning(self.ctx)

    def profile(self, on=True, classes=None):
        isdc_profile_enable(self.ctx, on, classes)

    def profile_read(self):
        return isdc_profile_read(self.ctx)

    def close(self):
        if self.ctx:
            isdc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
