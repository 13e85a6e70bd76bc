"""Continuous-batching request loop for ISDC integrations.

Requests (each one ISDC integration: dimension, side, nu, M, dt, steps and an
initial value) arrive over time.  A request is admitted into the batch engine
of its dimension as soon as the engine has a free slot and enough of its HBM
budget; its node state then stays on the device until its last step is done.
Every loop iteration ticks each engine that has running instances (one SDC
sweep for all of them, one CUDA graph launch); the 2D and 3D engines tick on
their own threads and streams, so their work overlaps on the GPU.  Latency of
a request = time its result is ready - its arrival time.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .isdc import ISDC_SLOT_FAILED, ISDC_SLOT_FINISHED, ISDC_SMOOTHER_JACOBI, ISDC_SMOOTHER_RBGS, Batch


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    ndim: int
    n: int
    nu: float
    M: int
    dt: float
    steps: int
    u0: np.ndarray
    admitted: float = -1.0
    done: float = -1.0
    result: np.ndarray | None = None
    sweeps: int = 0
    failed: bool = False


@dataclass
class ServeReport:
    requests: list = field(default_factory=list)
    wall_s: float = 0.0
    dof_sweeps: float = 0.0

    def latencies(self):
        return np.array([r.done - r.arrival for r in self.requests if r.done >= 0])

    def summary(self):
        lat = self.latencies()
        return {"requests": len(self.requests), "completed": int(len(lat)),
                "failed": int(sum(r.failed for r in self.requests)),
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_s": float(lat.mean()) if len(lat) else None,
                "wall_s": self.wall_s, "dof_sweeps_per_s": self.dof_sweeps / self.wall_s if self.wall_s else None}


class Server:
    """One batch engine per dimension: 2D damped Jacobi V(1,1), 3D red-black
    Gauss-Seidel V(2,2), L V-cycles, FP32 V-cycles with FP64 SDC state."""

    def __init__(self, hbm_budget_bytes=(96 << 30, 96 << 30), max_side=(1023, 255), max_M=5, n_vcycles=2,
                 tol=1e-10, max_sweeps=100):
        self.engines = {
            2: Batch(2, max_side[0], max_M, hbm_budget_bytes[0], n_vcycles, smoother=ISDC_SMOOTHER_JACOBI,
                     nu1=1, nu2=1, tol=tol, max_sweeps=max_sweeps),
            3: Batch(3, max_side[1], max_M, hbm_budget_bytes[1], n_vcycles, smoother=ISDC_SMOOTHER_RBGS,
                     nu1=2, nu2=2, tol=tol, max_sweeps=max_sweeps),
        }

    def run(self, requests: list[Request], realtime: bool = True) -> ServeReport:
        """Serve `requests` (sorted by arrival).  realtime=True admits a request
        only once the wall clock has reached its arrival time; False admits as
        fast as slots and memory allow (arrival times then only order them)."""
        pending = {2: [r for r in requests if r.ndim == 2], 3: [r for r in requests if r.ndim == 3]}
        report = ServeReport(requests=list(requests))
        t0 = time.perf_counter()
        lock = threading.Lock()
        dof = [0.0]

        def now():
            return time.perf_counter() - t0

        def worker(dim):
            eng = self.engines[dim]
            queue = pending[dim]
            live = {}  # slot -> request
            while queue or live:
                # admit everything that has arrived and fits
                while queue and (not realtime or queue[0].arrival <= now()):
                    r = queue[0]
                    slot = eng.admit(r.n, r.nu, r.M, r.dt, r.steps, r.u0)
                    if slot is None:
                        break
                    r.admitted = now()
                    live[slot] = r
                    queue.pop(0)
                if not live:
                    if queue:
                        time.sleep(max(0.0, min(0.002, queue[0].arrival - now())))
                    continue
                running, finished = eng.tick()
                with lock:
                    dof[0] += sum(float(r.n ** dim) for r in live.values())
                if finished:
                    for slot in list(live):
                        info = eng.query(slot)
                        if info.state in (ISDC_SLOT_FINISHED, ISDC_SLOT_FAILED):
                            r = live.pop(slot)
                            r.failed = info.state == ISDC_SLOT_FAILED
                            r.sweeps = info.total_sweeps
                            r.result = eng.take(slot)
                            r.done = now()

        threads = [threading.Thread(target=worker, args=(d,)) for d in (2, 3) if pending[d]]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        report.wall_s = now()
        report.dof_sweeps = dof[0]
        return report

    def close(self):
        for e in self.engines.values():
            e.close()
