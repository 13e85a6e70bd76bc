"""Full-size parity against the FP64 oracle run on all host cores.

The oracle's all-core build (the same C file with -fopenmp, bitwise equal to
the plain build; tests/test_oracle_threads.py) makes whole steps of the
full-size workloads affordable on the host, so the CUDA path is compared with
it element by element at the sizes the bench times:
  - 255^3, M = 5 Gauss-Lobatto, RB-GS V(2,2), L = 2 (Sec. 2 Eq. 4, Sec. 3):
    the FP64 path with the oracle's sweep count within rel L2 1e-12, its own
    until-tolerance sweep count within one of the oracle's (threshold ties),
    and the FP32-V-cycle path within rel L2 1e-9 at SDC residual < 1e-10;
  - 511^3 FP32 V-cycles (nu from seed 3), first step, within rel L2 1e-9;
  - the largest instance of the 256-instance batch against the oracle.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import make_gpu, to_dev
from isdc_inputs import initial_condition, workload_3d_255, workload_3d_511_mixed

pytestmark = pytest.mark.gpu
RB = O.SMOOTHER_RBGS


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def oracle_255():
    w = workload_3d_255()
    p = O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=w.nu1, nu2=w.nu2, max_sweeps=150)
    u0 = initial_condition(3, w.n, w.seed)
    with O.all_cores():
        r = O.isdc_step(p, u0, 0, w.n_vcycles)
    assert r.status == 0 and r.residuals[-1] < 1e-10
    return w, p, u0, r


def test_255_fp64_with_the_oracle_sweep_count(oracle_255):
    w, p, u0, r = oracle_255
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, r.sweeps, w.n_vcycles)
    got = u.cpu().numpy()
    g.close()
    err = rel_l2(got, r.u)
    print(f"255^3 FP64, {r.sweeps} sweeps: rel L2 {err:.3e}")
    assert err <= 1e-12


def test_255_fp64_until_tolerance_sweep_count(oracle_255):
    w, p, u0, r = oracle_255
    g = make_gpu(p)
    u = to_dev(u0)
    assert g.step(u, 0, w.n_vcycles) == 0
    sweeps, _ = g.stats()
    R = g.residual()
    g.close()
    print(f"255^3 FP64 until 1e-10: GPU {sweeps} sweeps (R {R:.3e}), oracle {r.sweeps} (R {r.residuals[-1]:.3e})")
    assert abs(sweeps - r.sweeps) <= 1 and R < 1e-10


def test_255_fp32_vcycles_one_step(oracle_255):
    w, p, u0, r = oracle_255
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(u0)
    assert g.step(u, 0, w.n_vcycles) == 0
    R = g.residual()
    got = u.cpu().numpy()
    g.close()
    err = rel_l2(got, r.u)
    print(f"255^3 FP32 V-cycles until 1e-10: rel L2 {err:.3e} vs the FP64 oracle (R {R:.3e})")
    assert R < 1e-10 and err <= 1e-9


def test_511_fp32_vcycles_first_step():
    w = workload_3d_511_mixed()
    p = O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=w.nu1, nu2=w.nu2, max_sweeps=200)
    u0 = initial_condition(3, w.n, w.seed)
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(u0)
    assert g.step(u, 0, w.n_vcycles) == 0
    R, (sweeps, _) = g.residual(), g.stats()
    got = u.cpu().numpy()
    g.close()
    del u
    with O.all_cores():
        r = O.isdc_step(p, u0, 0, w.n_vcycles)
    assert r.status == 0
    err = rel_l2(got, r.u)
    print(f"511^3 FP32 V-cycles step 1: rel L2 {err:.3e} vs the FP64 oracle; sweeps GPU {sweeps} "
          f"oracle {r.sweeps}; R GPU {R:.3e} oracle {r.residuals[-1]:.3e}")
    assert R < 1e-10 and err <= 1e-9


def test_511_fp32_vcycles_all_steps_satisfy_the_collocation_equations():
    """All 10 steps of the 511^3 FP32-V-cycle workload: after every step the
    oracle recomputes, in FP64 on all host cores, the SDC residual of the GPU's
    node values (the collocation equations of Sec. 2 evaluated at them; an
    element-wise oracle run of every step would take over an hour on the host).
    Each must be below the 1e-10 stopping tolerance and agree with the GPU's own
    residual to 1e-13 absolute; step 1 is compared element by element above."""
    w = workload_3d_511_mixed()
    p = O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=w.nu1, nu2=w.nu2, max_sweeps=200)
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(initial_condition(3, w.n, w.seed))
    for step in range(w.steps):
        assert g.step(u, 0, w.n_vcycles) == 0
        R = g.residual()
        sweeps, _ = g.stats()
        nodes = g.nodes().cpu().numpy()
        with O.all_cores():
            R_oracle = O.sdc_residual(p, nodes)
        del nodes
        print(f"511^3 FP32 V-cycles step {step + 1}: {sweeps} sweeps, R GPU {R:.3e}, R oracle {R_oracle:.3e}")
        assert R < 1e-10 and R_oracle < 1e-10 and abs(R_oracle - R) <= 1e-13, (step, R, R_oracle)
    assert bool(np.isfinite(u.cpu().numpy()).all())
    g.close()


def test_largest_batch_instance_against_the_oracle():
    """The 256-instance batch (one step each) at full size; its largest
    instance (side 1023) and its median one against the FP64 oracle."""
    import paper_1401_7824_gb300 as G
    from isdc_inputs import batch_instances
    insts = batch_instances(256, seed=4)
    eng = G.Batch(2, 1023, 5, 200 << 30, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150)
    slots = [eng.admit(w.n, w.nu, w.M, w.dt, 1, initial_condition(2, w.n, w.seed)) for w in insts]
    assert all(s is not None for s in slots)
    while eng.tick()[0]:
        pass
    order = sorted(range(len(insts)), key=lambda q: insts[q].n)
    sample = [order[-1], order[len(order) // 2]]
    results = {q: eng.take(slots[q]) for q in sample}
    eng.close()
    for q in sample:
        w = insts[q]
        p = O.Problem(2, w.n, w.nu, w.M, w.dt, smoother=O.SMOOTHER_JACOBI, max_sweeps=150)
        with O.all_cores():
            r = O.isdc_step(p, initial_condition(2, w.n, w.seed), 0, 2)
        assert r.status == 0
        err = rel_l2(results[q], r.u)
        print(f"batch instance side {w.n}, M {w.M}, nu {w.nu:.4f}: rel L2 {err:.3e} vs the FP64 oracle")
        assert err <= 1e-9
