"""Batched engine and continuous-batching server (isdc_batch_*): results
against the FP64 oracle and against the same integration run alone.

Tolerance: the engine runs FP32 V-cycles with FP64 node state, so results are
compared with the FP64 oracle at relative L2 1e-9 once every step has reached
SDC residual 1e-10.  Alone vs in the mix the per-point arithmetic is the same
(the work lists only change which block computes a point), so the results
must agree exactly."""
import numpy as np
import pytest

import oracle as O
from gpu_util import rel_l2, torch_cuda
from isdc_inputs import initial_condition

pytestmark = pytest.mark.gpu

PROBS_2D = [  # n, nu, M, dt, steps
    (63, 0.3, 3, 0.05, 2),
    (127, 0.05, 5, 0.02, 2),
    (31, 1.0, 5, 0.01, 3),
    (63, 0.01, 3, 0.1, 2),
]
PROBS_3D = [
    (31, 0.1, 5, 0.02, 2),
    (15, 0.5, 3, 0.05, 2),
]


def _engine(ndim, budget=8 << 30):
    import paper_1401_7824_gb300 as G
    torch_cuda()
    if ndim == 2:
        return G.Batch(2, 127, 5, budget, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150)
    return G.Batch(3, 31, 5, budget, 2, smoother=G.ISDC_SMOOTHER_RBGS, nu1=2, nu2=2, max_sweeps=150)


def _run(eng, probs, ndim, seed0):
    slots = []
    for q, (n, nu, M, dt, steps) in enumerate(probs):
        slots.append(eng.admit(n, nu, M, dt, steps, initial_condition(ndim, n, seed0 + q)))
    assert all(s is not None for s in slots)
    for _ in range(10000):
        running, _ = eng.tick()
        if running == 0:
            break
    out = []
    for s in slots:
        info = eng.query(s)
        assert info.state == 2, info.state
        out.append((eng.take(s), info.total_sweeps))
    return out


@pytest.mark.parametrize("ndim,probs", [(2, PROBS_2D), (3, PROBS_3D)])
def test_batch_matches_fp64_oracle(ndim, probs):
    eng = _engine(ndim)
    got = _run(eng, probs, ndim, 40)
    for q, (n, nu, M, dt, steps) in enumerate(probs):
        sm = O.SMOOTHER_JACOBI if ndim == 2 else O.SMOOTHER_RBGS
        nu1 = 1 if ndim == 2 else 2
        p = O.Problem(ndim, n, nu, M, dt, smoother=sm, nu1=nu1, nu2=nu1, max_sweeps=150)
        ref = O.integrate(p, initial_condition(ndim, n, 40 + q), steps, 0, 2)
        assert all(s == 0 for s in ref.status)
        assert rel_l2(got[q][0], ref.u) <= 1e-9, (q, rel_l2(got[q][0], ref.u))
    eng.close()


@pytest.mark.parametrize("depth", [-1, 0])
def test_batch_temporal_blocking_depths_match_fp64_oracle(depth):
    """2D damped-Jacobi V(1,1) engines with the sweep fused into the transfer
    passes (depth 1, the default) and with separate phases (depth 0), on sides
    with up to three grid-wide levels above the per-instance bottom block (511:
    levels 511, 255, 127, then 63 and below in one block) and bottom-only
    sides, against the FP64 oracle."""
    import paper_1401_7824_gb300 as G
    torch_cuda()
    probs = [(511, 0.05, 3, 0.02, 1), (255, 0.5, 5, 0.05, 1), (127, 0.02, 5, 0.1, 1), (63, 0.3, 3, 0.05, 2),
             (15, 1.0, 3, 0.01, 1)]
    eng = G.Batch(2, 511, 5, 16 << 30, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150,
                  temporal_blocking=depth)
    got = _run(eng, probs, 2, 110)
    info = eng.stats()
    assert info.fused == (1 if depth == -1 else 0) and info.bytes_last_tick > 0
    eng.close()
    for q, (n, nu, M, dt, steps) in enumerate(probs):
        p = O.Problem(2, n, nu, M, dt, smoother=O.SMOOTHER_JACOBI, max_sweeps=150)
        with O.all_cores():
            ref = O.integrate(p, initial_condition(2, n, 110 + q), steps, 0, 2)
        assert all(s == 0 for s in ref.status)
        assert rel_l2(got[q][0], ref.u) <= 1e-9, (q, rel_l2(got[q][0], ref.u))


@pytest.mark.parametrize("ndim", [2, 3])
def test_batch_every_node_count_matches_fp64_oracle(ndim):
    """The sweep end is compiled per node count (one work list per M): an
    engine with max_M = 7 holding instances with M = 2, 4, 6 and 7 (2D damped
    Jacobi, fused passes; 3D red-black with side 63, two grid-wide levels above
    the per-instance bottom block) against the FP64 oracle."""
    import paper_1401_7824_gb300 as G
    torch_cuda()
    if ndim == 2:
        probs = [(127, 0.2, 2, 0.05, 2), (255, 0.05, 4, 0.02, 1), (63, 0.5, 6, 0.05, 1), (127, 0.02, 7, 0.1, 1)]
        eng = G.Batch(2, 255, 7, 8 << 30, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150)
        sm, nu1 = O.SMOOTHER_JACOBI, 1
    else:
        probs = [(63, 0.1, 2, 0.05, 1), (63, 0.05, 4, 0.02, 1), (31, 0.5, 6, 0.05, 1), (15, 1.0, 7, 0.02, 1)]
        eng = G.Batch(3, 63, 7, 8 << 30, 2, smoother=G.ISDC_SMOOTHER_RBGS, nu1=2, nu2=2, max_sweeps=150)
        sm, nu1 = O.SMOOTHER_RBGS, 2
    got = _run(eng, probs, ndim, 170)
    eng.close()
    for q, (n, nu, M, dt, steps) in enumerate(probs):
        p = O.Problem(ndim, n, nu, M, dt, smoother=sm, nu1=nu1, nu2=nu1, max_sweeps=150)
        with O.all_cores():
            ref = O.integrate(p, initial_condition(ndim, n, 170 + q), steps, 0, 2)
        assert all(s == 0 for s in ref.status)
        assert rel_l2(got[q][0], ref.u) <= 1e-9, (q, rel_l2(got[q][0], ref.u))


def test_batch_rbgs_2d_matches_fp64_oracle():
    """2D red-black Gauss-Seidel V(2,2) engine (row-structured passes on the
    grid-wide levels 255 and 127, the levels from 63 down in one block per
    instance) against the FP64 oracle."""
    import paper_1401_7824_gb300 as G
    torch_cuda()
    probs = [(255, 0.05, 3, 0.02, 1), (127, 0.3, 5, 0.05, 2), (63, 1.0, 5, 0.01, 1)]
    eng = G.Batch(2, 255, 5, 8 << 30, 2, smoother=G.ISDC_SMOOTHER_RBGS, nu1=2, nu2=2, max_sweeps=150)
    got = _run(eng, probs, 2, 190)
    eng.close()
    for q, (n, nu, M, dt, steps) in enumerate(probs):
        p = O.Problem(2, n, nu, M, dt, smoother=O.SMOOTHER_RBGS, nu1=2, nu2=2, max_sweeps=150)
        ref = O.integrate(p, initial_condition(2, n, 190 + q), steps, 0, 2)
        assert all(s == 0 for s in ref.status)
        assert rel_l2(got[q][0], ref.u) <= 1e-9, (q, rel_l2(got[q][0], ref.u))


@pytest.mark.parametrize("ndim", [2, 3])
def test_batch_launch_shapes_give_identical_results(ndim):
    """An instance admitted into a fresh engine sweeps through the autotuner's
    trial ticks (every graph shape, in 2D damped Jacobi the persistent
    one-launch ticks, then 2 to 4 lanes), the same instance admitted after
    tuning sweeps in the chosen shape only, dealt to a lane beside another
    instance: the results agree bit for bit, so no launch form (nor the rows per
    tile of the red-black passes, nor the lane) changes the arithmetic."""
    import paper_1401_7824_gb300 as G
    torch_cuda()
    if ndim == 2:
        prob, warm_n = (255, 0.1, 5, 0.02, 1), 63

        def engine():
            return G.Batch(2, 255, 5, 8 << 30, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150)
    else:
        prob, warm_n = (63, 0.1, 5, 0.02, 1), 15

        def engine():
            return G.Batch(3, 63, 5, 8 << 30, 2, smoother=G.ISDC_SMOOTHER_RBGS, nu1=2, nu2=2, max_sweeps=150)

    fresh = engine()
    r_fresh = _run(fresh, [prob], ndim, 150)
    fresh.close()
    tuned = engine()
    warm = tuned.admit(warm_n, 0.5, 3, 0.05, 50, initial_condition(ndim, warm_n, 9))
    for _ in range(30):
        tuned.tick()
        if tuned.stats().tuned:
            break
    assert tuned.stats().tuned == 1
    r_tuned = _run_keep(tuned, [prob], ndim, 150, ignore=[warm])
    tuned.close()
    np.testing.assert_array_equal(r_fresh[0][0], r_tuned[0][0])
    assert r_fresh[0][1] == r_tuned[0][1]


def _run_keep(eng, probs, ndim, seed0, ignore=()):
    slots = [eng.admit(n, nu, M, dt, steps, initial_condition(ndim, n, seed0 + q))
             for q, (n, nu, M, dt, steps) in enumerate(probs)]
    assert all(s is not None for s in slots)
    for _ in range(10000):
        eng.tick()
        if all(eng.query(s).state != 1 for s in slots):
            break
    out = []
    for s in slots:
        info = eng.query(s)
        assert info.state == 2, info.state
        out.append((eng.take(s), info.total_sweeps))
    return out


@pytest.mark.parametrize("ndim", [2, 3])
def test_batch_alone_equals_in_the_mix(ndim):
    """Each instance of a mix gives the same result bit for bit as when it runs
    alone: in the mix it shares work lists and launches with the others and,
    once the autotuner tries 2 to 4 lanes, is dealt to one of several
    concurrent chains of the tick graph (3D: red-black row-structured passes)."""
    probs = PROBS_2D if ndim == 2 else PROBS_3D + [(31, 0.3, 3, 0.05, 1), (31, 0.02, 5, 0.1, 1)]
    mix = _engine(ndim)
    together = _run(mix, probs, ndim, 70)
    mix.close()
    for q, prob in enumerate(probs):
        alone_eng = _engine(ndim)
        alone = _run(alone_eng, [prob], ndim, 70 + q)
        alone_eng.close()
        np.testing.assert_array_equal(alone[0][0], together[q][0])
        assert alone[0][1] == together[q][1]


def test_grid_barrier_wait_is_bounded_and_reported():
    """The one-launch tick's grid barrier never waits without bound: when the
    arrivals it expects never come (phantom blocks), every block's wait ends
    after the limit, the failure is reported to the host, and the device is
    still usable (failure detection without a GPU fault)."""
    import ctypes
    import time
    import paper_1401_7824_gb300 as G
    torch_cuda()
    lib = G.load()
    failed = ctypes.c_int(-1)
    assert lib.isdc_batch_barrier_selftest(152, 0, 1.0, ctypes.byref(failed)) == G.ISDC_OK and failed.value == 0
    t0 = time.perf_counter()
    assert lib.isdc_batch_barrier_selftest(152, 1, 0.05, ctypes.byref(failed)) == G.ISDC_OK and failed.value == 1
    assert time.perf_counter() - t0 < 5.0
    assert lib.isdc_batch_barrier_selftest(152, 0, 1.0, ctypes.byref(failed)) == G.ISDC_OK and failed.value == 0
    eng = _engine(2)  # and an engine still runs
    got = _run(eng, PROBS_2D[:1], 2, 40)
    eng.close()
    assert np.isfinite(got[0][0]).all()


def test_batch_budget_admission_is_soft():
    import paper_1401_7824_gb300 as G
    eng = _engine(2, budget=1)
    assert eng.admit(63, 0.1, 3, 0.05, 1, initial_condition(2, 63, 1)) is None
    eng.close()
    u = initial_condition(2, 127, 2)
    probe = _engine(2)
    one = probe.query(probe.admit(127, 0.1, 5, 0.02, 1, u)).device_bytes
    probe.close()
    # room for exactly one 127^2, M = 5 instance: the second waits until the first is taken
    eng = _engine(2, budget=int(1.5 * one))
    s1 = eng.admit(127, 0.1, 5, 0.02, 1, u)
    assert s1 is not None
    assert eng.admit(127, 0.1, 5, 0.02, 1, u) is None
    while eng.tick()[0]:
        pass
    eng.take(s1)
    assert eng.admit(127, 0.1, 5, 0.02, 1, u) is not None
    assert eng.stats().tuned in (0, 1)
    with pytest.raises(G.IsdcError):
        eng.admit(255, 0.1, 3, 0.02, 1, initial_condition(2, 255, 3))  # beyond max_side
    eng.close()


def test_server_continuous_batching_same_alone_and_in_mix():
    from paper_1401_7824_gb300.serve import Request, Server
    reqs = []
    specs = [(2, 63, 0.3, 3, 0.05, 2), (3, 15, 0.5, 3, 0.05, 2), (2, 127, 0.05, 5, 0.02, 1),
             (3, 31, 0.1, 5, 0.02, 1), (2, 31, 1.0, 5, 0.01, 2)]
    for q, (d, n, nu, M, dt, steps) in enumerate(specs):
        reqs.append(Request(q, 0.01 * q, d, n, nu, M, dt, steps, initial_condition(d, n, 90 + q)))
    srv = Server(hbm_budget_bytes=(4 << 30, 4 << 30), max_side=(127, 31))
    rep = srv.run(reqs, realtime=True)
    srv.close()
    s = rep.summary()
    assert s["completed"] == len(specs) and s["failed"] == 0
    assert s["p99_s"] >= s["p50_s"] > 0
    for q, (d, n, nu, M, dt, steps) in enumerate(specs):
        alone = Server(hbm_budget_bytes=(4 << 30, 4 << 30), max_side=(127, 31))
        r1 = alone.run([Request(q, 0.0, d, n, nu, M, dt, steps, initial_condition(d, n, 90 + q))])
        alone.close()
        np.testing.assert_array_equal(r1.requests[0].result, reqs[q].result)


def test_server_queues_requests_under_memory_pressure():
    """With room for one instance at a time, requests wait for memory, every
    request still completes, and results equal the runs alone."""
    from paper_1401_7824_gb300.serve import Request, Server
    probe = _engine(2)
    one = probe.query(probe.admit(63, 0.1, 5, 0.02, 1, initial_condition(2, 63, 1))).device_bytes
    probe.close()
    specs = [(63, 0.3, 5, 0.05, 1), (63, 0.05, 5, 0.02, 1), (63, 1.0, 3, 0.01, 2)]
    reqs = [Request(q, 0.0, 2, n, nu, M, dt, steps, initial_condition(2, n, 130 + q))
            for q, (n, nu, M, dt, steps) in enumerate(specs)]
    srv = Server(hbm_budget_bytes=(int(1.2 * one), 1 << 30), max_side=(63, 15))
    rep = srv.run(reqs, realtime=False)
    srv.close()
    assert rep.summary()["completed"] == 3
    admitted = sorted(r.admitted for r in reqs)
    done = sorted(r.done for r in reqs)
    assert admitted[1] >= done[0] and admitted[2] >= done[1]   # one at a time
    for q, (n, nu, M, dt, steps) in enumerate(specs):
        alone = Server(hbm_budget_bytes=(4 << 30, 1 << 30), max_side=(63, 15))
        r1 = alone.run([Request(q, 0.0, 2, n, nu, M, dt, steps, initial_condition(2, n, 130 + q))])
        alone.close()
        np.testing.assert_array_equal(r1.requests[0].result, reqs[q].result)


def test_full_256_instance_batch_matches_single_instance_runs():
    """The 256-instance batch at full size (one step each): sampled instances
    (smallest, median and largest side) against independent single-instance
    runs with FP32 V-cycles, both at SDC residual < 1e-10."""
    import paper_1401_7824_gb300 as G
    from gpu_util import make_gpu, to_dev
    from isdc_inputs import batch_instances
    insts = batch_instances(256, seed=4)
    eng = G.Batch(2, 1023, 5, 200 << 30, 2, smoother=G.ISDC_SMOOTHER_JACOBI, nu1=1, nu2=1, max_sweeps=150)
    slots = [eng.admit(w.n, w.nu, w.M, w.dt, 1, initial_condition(2, w.n, w.seed)) for w in insts]
    assert all(s is not None for s in slots)
    while eng.tick()[0]:
        pass
    order = sorted(range(len(insts)), key=lambda q: insts[q].n)
    sample = {order[0], order[len(order) // 2], order[-1]}
    results = {}
    for q, s in enumerate(slots):
        info = eng.query(s)
        assert info.state == G.ISDC_SLOT_FINISHED and info.nonconverged_steps == 0
        out = eng.take(s)
        if q in sample:
            results[q] = out
    eng.close()
    for q in sample:
        w = insts[q]
        p = O.Problem(2, w.n, w.nu, w.M, w.dt, smoother=O.SMOOTHER_JACOBI, max_sweeps=150)
        g = make_gpu(p, vcycle_fp32=True)
        u = to_dev(initial_condition(2, w.n, w.seed))
        assert g.step(u, 0, 2) == 0
        assert rel_l2(results[q], u.cpu().numpy()) <= 1e-9
        g.close()
