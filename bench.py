#!/usr/bin/env python
"""Benchmark of the GB300 ISDC hot path.

One bench step = one ISDC time step of the workload (Sec. 2 Eq. 4, Sec. 3):
spread, SDC sweeps with L V-cycles per node solve until the max-norm SDC
residual is below 1e-10, u <- u_M.  Metric: DOF-sweeps/s = (interior points)
x (sweeps executed) / wall time, whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on host cores)

Multi-GPU (torchrun, one rank per GPU): every rank integrates its own copy of
the workload (independent replicas, no collective on the data path), weak
scaling.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import isdc_inputs as W  # noqa: E402

FP64_OPS_PER_SM_CLK = 2      # nominal FP64 issue per SM per clock (used only when the probe cannot run)
FP32_OPS_PER_SM_CLK = 128
SMS = 152
SM_MAX_MHZ = 2070.0
L2_BYTES = 129 * 2 ** 20


def workloads():
    return {
        "3d_n255_M5_fp64": W.workload_3d_255(),
        "3d_n255_M5_mixed": W.Workload("3d_n255_M5_mixed", 3, 255, 0.1, 5, 0.02, 20, 2, 1, 2, 2,
                                       vcycle_fp32=True, seed=2),
        "3d_n511_M5_mixed": W.workload_3d_511_mixed(),
        "2d_n127_M3_fp64": W.workload_2d_127(),
        "3d_n255_M5_radau_fp64": W.workload_3d_255_radau(),
        "3d_n255_M5_legendre_fp64": W.workload_3d_255_legendre(),
        "2d_n1023_M5_compact_fp64": W.workload_2d_1023_compact(),
        "2d_n1024_M5_burgers_fp64": W.workload_2d_1024_burgers(),
    }


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


SDC_CLASSES = ("spread", "eval_f", "rhs", "sweep_end", "resnorm")  # kernels in csrc/sdc_kernels.cuh


def kernel_source_sha(cls: str) -> str:
    """sha256 prefix of the header that holds the kernels of class cls."""
    name = "sdc_kernels.cuh" if cls in SDC_CLASSES else "kernels.cuh"
    with open(os.path.join(ROOT, "paper_1401_7824_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(workload: str, cls: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (profiles/ncu_traffic.txt: workload class sha bytes,
    sha of the header holding that class's kernels)."""
    sha = kernel_source_sha(cls)
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")) as f:
            for line in f:
                p = line.split()
                if len(p) == 4 and not line.startswith("#") and p[0] == workload and p[1] == cls and p[2] == sha:
                    return float(p[3])
    except OSError:
        pass
    return None


def roofline(prof: dict, dom: str, workload: str, shares: dict, peak: dict | None = None):
    """Roofline of kernel class `dom`: algorithmic bytes / ops per launch over
    its event-timed average launch duration in the timed region.  FP64-bound
    classes are reported against the FP64 issue rate measured in this run."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    r = prof[dom]
    per_launch_s = r["total_ms"] / 1e3 / r["launches"]
    bytes_l = r["bytes"] / r["launches"]
    dp_l = r["fp64_ops"] / r["launches"]
    sp_l = r["fp32_ops"] / r["launches"]
    dp_peak = peak["ops_per_s"] if peak else SMS * FP64_OPS_PER_SM_CLK * SM_MAX_MHZ * 1e6
    sp_peak = SMS * FP32_OPS_PER_SM_CLK * SM_MAX_MHZ * 1e6
    t_hbm = bytes_l / (hbm * 1e9)
    t_dp = dp_l / dp_peak
    t_sp = sp_l / sp_peak
    out = {"kernel": dom, "launches": r["launches"], "us_per_launch": per_launch_s * 1e6,
           "algorithmic_bytes_per_launch": bytes_l, "fp64_ops_per_launch": dp_l, "fp32_ops_per_launch": sp_l}
    if t_hbm >= max(t_dp, t_sp):
        ach = bytes_l / per_launch_s / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                   peak_source=f"{hbm_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)")
    elif t_dp >= t_sp:
        ach = dp_l / per_launch_s / 1e12
        out.update(bound="alu", achieved=ach, peak=dp_peak / 1e12, unit="T FP64-op/s", frac=ach / (dp_peak / 1e12),
                   peak_source=("measured in this run: FP64 FMA issue probe (libisdc_probe.so)" if peak else
                                "derived: 152 SMs x 2 FP64 add/mul/FMA per SM-clock x 2070 MHz"),
                   hbm_frac=bytes_l / per_launch_s / 1e9 / hbm)
    else:
        ach = sp_l / per_launch_s / 1e12
        out.update(bound="alu", achieved=ach, peak=sp_peak / 1e12, unit="T FP32-op/s", frac=ach / (sp_peak / 1e12),
                   peak_source="derived: 152 SMs x 128 FP32 lanes x 2070 MHz",
                   hbm_frac=bytes_l / per_launch_s / 1e9 / hbm)
    out["traffic"] = traffic_for(workload, dom)
    out["shares"] = shares
    return out


def class_shares(prof: dict):
    total = sum(v["total_ms"] for v in prof.values() if v["total_ms"] > 0)
    return {k: round(v["total_ms"] / total, 4)
            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["total_ms"]) if v["total_ms"] > 0}


def oracle_sweep_rate(w, n_override=None, sweeps=1):
    """DOF-sweeps/s of the FP64 CPU oracle on one SDC sweep of the workload
    (single-threaded plain C)."""
    import oracle as O
    n = n_override or w.n
    p = O.Problem(w.ndim, n, w.nu, w.M, w.dt, smoother=w.smoother, nu1=w.nu1, nu2=w.nu2, omega=w.omega,
                  reaction=w.reaction, nodes=w.nodes, stencil=w.stencil, equation=w.equation)
    u0 = W.periodic_bump(w.ndim, n, w.seed) if w.equation == 1 else W.initial_condition(w.ndim, n, w.seed)
    O.build()
    t0 = time.perf_counter()
    O.isdc_step(p, u0, sweeps, w.n_vcycles)
    dt = time.perf_counter() - t0
    return n ** w.ndim * sweeps / dt, dt, n


def run_reference(args):
    """The oracle as it stands (its all-core build, every host core) on the
    workload's own grid: each step one SDC sweep of step 1 of the workload."""
    import oracle as O
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    w = workloads().get(args.workload, W.workload_3d_255())
    with O.all_cores():
        cores = O.threads()
        for _ in range(args.warmup):
            oracle_sweep_rate(w)
        total_dof_sweeps, total_t = 0.0, 0.0
        for _ in range(args.steps):
            rate, dt, n = oracle_sweep_rate(w)
            total_dof_sweeps += n ** w.ndim
            total_t += dt
    value = total_dof_sweeps / total_t
    solves = w.M - (1 if w.nodes == 0 else 0)
    sample = (f"each step: 1 SDC sweep ({solves} node solves x {w.n_vcycles} V-cycles + residual) of step 1 of "
              f"the workload on its own {w.n}^{w.ndim} grid, from its seeded initial state, all-core oracle "
              f"build on {cores} threads")
    line = {"metric": "DOF-sweeps/s", "value": value, "unit": "DOF-sweeps/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": "DOF-sweeps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOF-sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def combine_ranks(times, work, world, device):
    """Whole-job figures of independent replicas: the slowest rank's times
    (max over ranks) and the work of all ranks (sum).  No data-path collective:
    this is the only cross-rank exchange, after the timed region."""
    if world <= 1:
        return list(times), list(work)
    import torch
    import torch.distributed as dist
    t = torch.tensor(times, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor(work, dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return [float(v) for v in t], [float(v) for v in w]


def config_of(w):
    N = w.n ** w.ndim
    P = w.M if w.nodes == 0 else w.M + 1  # points of a sweep: t_0 and the nodes
    state_bytes = 4 * P * N * 8  # U, F, f^E (P arrays each), C (P - 1), beta (1), FP64
    return {"workload": w.name, "ndim": w.ndim, "n": w.n, "dofs": N, "M": w.M,
            "nodes": ["gauss-lobatto", "gauss-radau-right", "gauss-legendre"][w.nodes],
            "equation": "viscous Burgers, periodic, WENO5 advection" if w.equation == 1
            else "u_t = nu Lap u + f^E(u), Dirichlet",
            "stencil": "4th-order compact with W" if w.stencil == 1 else ("5-point" if w.ndim == 2 else "7-point"),
            "nu": w.nu, "dt": w.dt, "L_vcycles": w.n_vcycles,
            "smoother": ("rbgs" if w.smoother == 1 else "wjacobi") + f" V({w.nu1},{w.nu2})",
            "reaction": "u-u^3" if (w.reaction == 1 and w.equation == 0) else "none",
            "tol": w.tol, "vcycle_precision": "fp32" if w.vcycle_fp32 else "fp64",
            "l2": f"inputs larger than L2 (node state {state_bytes / 1e9:.2f} GB > {L2_BYTES / 1e6:.0f} MB L2)"
            if state_bytes > L2_BYTES else "inputs fit in L2 (latency-bound case)",
            "parallelism": "replicas (one independent instance per GPU)"}


def fp64_peak():
    """The GPU's FP64 issue rate measured in this run (libisdc_probe.so: independent
    FMA chains on every SM; one FMA = one FP64 operation), in operations per second."""
    import paper_1401_7824_gb300 as G
    ops, ms = G.probe_fp64_rate()
    return {"ops_per_s": ops, "probe_ms": ms,
            "per_sm_clock_at_max": ops / (SMS * SM_MAX_MHZ * 1e6)}


def latency_record(prof_full, shares, dom, elapsed, sweeps_total, launches):
    """Roofline record of a workload whose node state fits in L2: the time per
    sweep and the launches per sweep (no bandwidth or ALU bound applies)."""
    us = elapsed / max(1, sweeps_total) * 1e6
    return {"bound": "latency", "achieved": us, "unit": "us/sweep", "peak": None, "frac": None,
            "launches_per_sweep": launches / max(1, sweeps_total), "us_per_sweep": us,
            "kernel": dom, "traffic": None, "shares": shares}


def measure(w, args, world, barrier, peak):
    """Time K until-tolerance steps of workload w on this rank (inputs resident
    on the device), then the same through the host-buffer entry point."""
    import torch
    import paper_1401_7824_gb300 as G
    N = w.n ** w.ndim
    u0 = W.workload_initial(w)
    g = G.Isdc(w.ndim, w.n, w.nu, w.M, w.dt, smoother=w.smoother, nu1=w.nu1, nu2=w.nu2, omega=w.omega,
               vcycle_fp32=w.vcycle_fp32, tol=w.tol, max_sweeps=200, temporal_blocking=args.temporal_blocking,
               fused_transfer=args.fused_transfer, rb_run=args.rb_run, use_graphs=args.use_graphs,
               nodes=w.nodes, stencil=w.stencil, equation=w.equation,
               reaction=G.ISDC_REACTION_ALLEN_CAHN if w.reaction == 1 else G.ISDC_REACTION_NONE)
    stream = torch.cuda.current_stream()
    u = torch.from_numpy(u0).cuda()
    for _ in range(args.warmup):
        g.step(u, 0, w.n_vcycles)
    torch.cuda.synchronize()
    # one untimed step with every kernel class event-timed: the per-class shares
    # and the dominant class (timed alone inside the measured region below)
    g.profile(True)
    g.step(u, 0, w.n_vcycles)
    full_prof = g.profile_read()
    g.profile(False)
    shares = class_shares(full_prof)
    dominant = next(iter(shares))

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    clocks.start()
    g.profile(True, classes=[])  # launch counts only: no events, no synchronisation
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps, vcycles, statuses = [], [], []
    e0.record(stream)
    for _ in range(args.steps):
        statuses.append(g.step(u, 0, w.n_vcycles))
        s, v = g.stats()
        sweeps.append(s)
        vcycles.append(v)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = int(sum(v["launches"] for v in g.profile_read().values()))
    g.profile(False)
    # the dominant class's launches timed with CUDA events on the library's
    # stream over a second timed region of the same length (the event read-back
    # after every sweep would slow a latency-bound workload's first region)
    profiled_elapsed = None
    prof = full_prof
    if not args.no_profile:
        g.profile(True, classes=[dominant])
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            g.step(u, 0, w.n_vcycles)
        e1.record(stream)
        torch.cuda.synchronize()
        profiled_elapsed = e0.elapsed_time(e1) / 1e3
        prof = g.profile_read()
        g.profile(False)
    clk = clocks.stop()
    residual = g.residual()
    dof_sweeps = float(N * sum(sweeps))

    # end to end through the public C ABI with host buffers: H2D + step + D2H each step
    uh = torch.from_numpy(u0).pin_memory()
    g.step_host(uh.numpy(), 0, w.n_vcycles)  # first call allocates the device staging buffer
    barrier()
    t0 = time.perf_counter()
    e2e_sweeps = 0
    for _ in range(args.steps):
        g.step_host(uh.numpy(), 0, w.n_vcycles)
        e2e_sweeps += g.stats()[0]
    e2e_t = time.perf_counter() - t0
    barrier()
    tuning = g.tuning()
    g.close()
    del u, uh
    torch.cuda.empty_cache()

    (elapsed, e2e_t), (dof_sweeps, e2e_work) = combine_ranks([elapsed, e2e_t], [dof_sweeps, float(N * e2e_sweeps)],
                                                             world, "cuda")
    cfg = config_of(w)
    if cfg["l2"].startswith("inputs fit"):
        roof = latency_record(full_prof, shares, dominant, elapsed, world * sum(sweeps), world * launches)
    else:
        roof = roofline(prof, dominant, w.name, shares, peak)
    return {
        "value": dof_sweeps / elapsed, "elapsed": elapsed, "config": cfg,
        "ms_per_step": elapsed / args.steps * 1e3, "steps_per_s": world * args.steps / elapsed,
        "sweeps_per_step": sweeps, "vcycles_per_step": vcycles, "residual_last_step": residual,
        "converged": all(s == 0 for s in statuses), "gpu_launches": launches, "roofline": roof,
        "profiled_region_ms_per_step": profiled_elapsed / args.steps * 1e3 if profiled_elapsed else None,
        "autotune": tuning, "clocks": clk,
        "e2e": {"value": e2e_work / e2e_t, "unit": "DOF-sweeps/s", "h2d_bytes_per_step": N * 8,
                "d2h_bytes_per_step": N * 8},
    }


def cpu_baseline(w):
    """The oracle as it stands, on one SDC sweep of step 1 of the workload: its
    all-core build (every host core) and its plain single-threaded build."""
    import oracle as O
    with O.all_cores():
        rate_all, dt_all, n = oracle_sweep_rate(w)
        cores = O.threads()
    rate_1, dt_1, _ = oracle_sweep_rate(w)
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines() if ln.startswith("Model name")), "")
    except Exception:
        pass
    solves = w.M - (1 if w.nodes == 0 else 0)
    return {"value": rate_all, "unit": "DOF-sweeps/s", "cores": cores, "kind": "oracle",
            "sample": f"1 SDC sweep of step 1 of the workload ({n}^{w.ndim} grid, {solves} node solves x "
                      f"{w.n_vcycles} V-cycles + residual): {dt_all:.2f} s on {cores} threads (all-core build), "
                      f"{dt_1:.1f} s single-threaded (plain build)",
            "single_core_value": rate_1, "nproc": os.cpu_count(), "cpu_model": model}


def run_ours(args):
    import dataclasses
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    peak = fp64_peak()
    w = workloads()[args.workload]
    m = measure(w, args, world, barrier, peak)
    line = {
        "metric": "DOF-sweeps/s", "value": m["value"], "unit": "DOF-sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not w.vcycle_fp32 else "f64 (FP32 V-cycles)",
        "data": "synthetic (seeded " + ("periodic Gaussian" if w.equation == 1 else "sin-mode") +
                " initial data + N(0, 0.01^2) noise)",
        "config": m["config"],
    }
    for k in ("steps_per_s", "sweeps_per_step", "vcycles_per_step", "residual_last_step", "converged",
              "gpu_launches", "roofline", "profiled_region_ms_per_step", "autotune", "clocks", "e2e"):
        line[k] = m[k]
    line["fp64_peak_probe"] = peak
    # the FP32-V-cycle forms of the workload (and the largest single-GPU one),
    # timed the same way, beside the FP64 headline
    if world == 1 and not args.no_extras and w.name == "3d_n255_M5_fp64":
        extras = {"fp32_vcycles": dataclasses.replace(w, name="3d_n255_M5_mixed", vcycle_fp32=True),
                  "n511_fp32_vcycles": W.workload_3d_511_mixed()}
        for key, we in extras.items():
            me = measure(we, args, world, barrier, peak)
            line[key] = {"workload": we.name, "value": me["value"], "unit": "DOF-sweeps/s",
                         "vs_headline": me["value"] / m["value"], "ms_per_step": me["ms_per_step"],
                         "steps": args.steps, "sweeps_per_step": me["sweeps_per_step"],
                         "residual_last_step": me["residual_last_step"], "converged": me["converged"],
                         "gpu_launches": me["gpu_launches"], "e2e": me["e2e"], "roofline": me["roofline"],
                         "clocks": me["clocks"], "config": me["config"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """batch_2d_256: 256 independent 2D instances (sides 2^j - 1, j in 6..10;
    nu, dt, M drawn from seed 4), damped Jacobi V(1,1).  batch_3d_32: 32
    independent 3D instances (sides 63..255, seed 6), red-black Gauss-Seidel
    V(2,2).  One batch engine each: FP32 V-cycles, FP64 SDC state, L = 2.  One
    bench step = one tick = one SDC sweep of every running instance (one CUDA
    graph launch).  Warm-up ticks include the autotuner's trial ticks."""
    import torch
    import paper_1401_7824_gb300 as G

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ndim = 3 if args.workload.startswith("batch_3d") else 2
    if ndim == 2:
        insts = W.batch_instances(args.instances, seed=4)
    else:
        insts = W.batch_instances_3d(min(args.instances, 32), seed=6)
    stream = torch.cuda.Stream()
    o = G.isdc_default_options()
    if ndim == 2:
        o.smoother, o.nu1, o.nu2 = G.ISDC_SMOOTHER_JACOBI, 1, 1
    else:
        o.smoother, o.nu1, o.nu2 = G.ISDC_SMOOTHER_RBGS, 2, 2
    o.vcycle_fp32, o.tol, o.max_sweeps = 1, 1e-10, 150
    o.temporal_blocking = -1 if args.temporal_blocking < 0 else min(args.temporal_blocking, 1)
    o.use_graphs = args.use_graphs
    import ctypes
    o.stream = ctypes.c_void_p(stream.cuda_stream)
    eng = G.isdc_batch_create(ndim, 1023 if ndim == 2 else 255, 5, 200 << 30, 2, o)
    sides = {}
    for q, w in enumerate(insts):
        slot = G.isdc_batch_admit(eng, w.n, w.nu, w.M, w.dt, w.steps, W.initial_condition(ndim, w.n, w.seed))
        assert slot is not None
        sides[slot] = w.n
    # warm-up: the requested ticks, and at least until the autotuner has kept a shape
    warm = 0
    while warm < args.warmup or (not G.isdc_batch_stats(eng).tuned and warm < 64):
        G.isdc_batch_tick(eng)
        warm += 1
    info = G.isdc_batch_stats(eng)
    launches0 = info.kernel_launches
    torch.cuda.synchronize()
    clocks = ClockSampler(None)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dofs = 0.0
    tick_bytes = 0.0
    e0.record(stream)
    for _ in range(args.steps):
        live = [s for s in sides if G.isdc_batch_query(eng, s).state == G.ISDC_SLOT_RUNNING]
        dofs += sum(float(sides[s] ** ndim) for s in live)
        G.isdc_batch_tick(eng)
        tick_bytes += G.isdc_batch_stats(eng).bytes_last_tick  # host-side counter, no device work
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    info = G.isdc_batch_stats(eng)
    launches = info.kernel_launches - launches0
    G.isdc_batch_destroy(eng)
    line = {"metric": "DOF-sweeps/s", "value": dofs / elapsed, "unit": "DOF-sweeps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": warm, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 V-cycles)",
            "data": "synthetic (seeded)",
            "config": {"workload": f"batch_{ndim}d_{len(insts)}",
                       "instances": len(insts),
                       "dofs_total": int(sum(w.n ** ndim for w in insts)),
                       "sides": "2^j - 1, j uniform in " + ("6..10" if ndim == 2 else "6..8"),
                       "smoother": "wjacobi V(1,1)" if ndim == 2 else "rbgs V(2,2)", "L_vcycles": 2,
                       "vcycle_precision": "fp32", "tol": 1e-10,
                       "l2": "inputs larger than L2 (all instances resident, tens of GB)",
                       "launch_shape": {"threads_per_block": info.threads_per_block,
                                        "blocks_per_sm": info.blocks_per_sm, "tuned": info.tuned}},
            "gpu_launches": int(launches),
            "clocks": clk}
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ach = tick_bytes / elapsed / 1e9
    line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "traffic": None, "kernel": "whole tick",
                        "algorithmic_bytes_per_tick": tick_bytes / args.steps,
                        "peak_source": ("measured" if "hbm_gbs" in peaks else "fallback") +
                                       " HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                        "note": "algorithmic bytes of every phase of the tick (each input read once, each output "
                                "written once) over the tick time; the FP64 phases (right-hand sides, sweep end) "
                                "are bound by FP64 issue, so the whole tick stays below the HBM bound"}
    line["config"]["fused_smoother"] = int(info.fused)
    line["config"]["kernels_per_tick"] = int(info.kernels_per_tick)
    line["config"]["launch_shape"]["lanes"] = int(info.lanes)
    line["config"]["launch_shape"]["lane_split"] = int(info.lane_split)
    if args.compare_fp64:
        # the same instances one at a time through the FP64 single-instance path
        tot_dofs, tot_t = 0.0, 0.0
        for w in insts[:args.compare_fp64]:
            g = G.Isdc(ndim, w.n, w.nu, w.M, w.dt, smoother=o.smoother, nu1=o.nu1, nu2=o.nu2, max_sweeps=150)
            u = torch.from_numpy(W.initial_condition(ndim, w.n, w.seed)).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step(u, 0, 2)
            torch.cuda.synchronize()
            tot_t += time.perf_counter() - t0
            tot_dofs += w.n ** ndim * g.stats()[0]
            g.close()
        line["fp64_single_instance"] = {"value": tot_dofs / tot_t, "unit": "DOF-sweeps/s",
                                        "instances": args.compare_fp64,
                                        "what": "first time step of each instance, FP64 V-cycles, one "
                                                "instance at a time through isdc_step"}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson stream of ISDC requests (70 % 2D sides 127..1023, 30 % 3D sides
    63..255, M in {3,5}, 10 steps, tol 1e-10) served by continuous batching."""
    import torch
    from paper_1401_7824_gb300.serve import Request, Server

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = W.request_stream(args.requests, rate=args.rate, seed=5)
    reqs = [Request(q, t, w.ndim, w.n, w.nu, w.M, w.dt, w.steps, W.initial_condition(w.ndim, w.n, w.seed))
            for q, (t, w) in enumerate(stream)]
    srv = Server(hbm_budget_bytes=(60 << 30, 160 << 30), max_side=(1023, 255))
    clocks = ClockSampler(None)
    clocks.start()
    rep = srv.run(reqs, realtime=True)
    clk = clocks.stop()
    srv.close()
    s = rep.summary()
    line = {"metric": "DOF-sweeps/s", "value": s["dof_sweeps_per_s"], "unit": "DOF-sweeps/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 0, "ms_per_step": s["wall_s"] * 1e3 / max(1, args.requests),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FP32 V-cycles)",
            "data": "synthetic Poisson request stream (seed 5)",
            "config": {"workload": "serve_poisson", "requests": args.requests, "rate_per_s": args.rate,
                       "mix": "70% 2D n in 127..1023, 30% 3D n in 63..255, M in {3,5}, 10 steps, tol 1e-10"},
            "latency": {"p50_s": s["p50_s"], "p99_s": s["p99_s"], "mean_s": s["mean_s"],
                        "completed": s["completed"], "failed": s["failed"], "wall_s": s["wall_s"]},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="3d_n255_M5_fp64",
                    choices=sorted(workloads()) + ["batch_2d_256", "batch_3d_32", "serve_poisson"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the FP32-V-cycle 255^3 and 511^3 lines")
    ap.add_argument("--probe-fp64", action="store_true", help="print the FP64 issue-rate probe and exit")
    ap.add_argument("--no-profile", action="store_true",
                    help="no per-launch events in the timed region (sweeps replay CUDA graphs); the roofline then "
                         "comes from the untimed fully profiled step")
    ap.add_argument("--compare-fp64", type=int, default=0, help="batch: also time N instances on the FP64 path")
    ap.add_argument("--instances", type=int, default=256,
                    help="batch: number of instances (the first K of the seeded 256 2D or 32 3D; smaller for "
                         "profiling)")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--fused-transfer", type=int, default=-1, choices=[-1, 0, 1],
                    help="residual + restriction: -1 tuned per level, 0 two launches, 1 one fused launch")
    ap.add_argument("--use-graphs", type=int, default=1, choices=[0, 1, 2],
                    help="sweeps replayed from CUDA graphs: 1 with programmatic dependencies, 2 ordinary, 0 none")
    ap.add_argument("--rb-run", type=int, default=0, choices=[0, 1, 2, 4, 8, 16, 32, -1, -2, -4, -8],
                    help="3D red-black run form of the natural-layout levels: 0 tuned")
    ap.add_argument("--temporal-blocking", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="3D FP32 red-black fine level: -1 autotuned, 0 one pass per colour, "
                         "1/2 red-black sweeps per blocked pass")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.probe_fp64:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        clocks = ClockSampler(None)
        clocks.start()
        r = [fp64_peak() for _ in range(5)]
        print(json.dumps({"fp64_probe": r, "clocks": clocks.stop()}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batch_2d_256", "batch_3d_32"):
        run_batch(args)
    elif args.workload == "serve_poisson":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
