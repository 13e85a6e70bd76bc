"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 path relative L2 <= 1e-12 per step;
FP32-V-cycle path relative L2 <= 1e-9 once both reach SDC residual <= 1e-10."""
import numpy as np
import pytest

import oracle as O
from gpu_util import make_gpu, rel_l2, to_dev
from isdc_inputs import initial_condition, workload_2d_127, workload_3d_255

pytestmark = pytest.mark.gpu

J, RB = O.SMOOTHER_JACOBI, O.SMOOTHER_RBGS


# --- V-cycles on one implicit Euler system (Sec. 3) ---------------------------
VCYCLE_CASES = [
    # ndim, n, smoother, nu1, nu2, a
    (2, 63, J, 1, 1, 0.01),
    (2, 127, RB, 2, 2, 0.003),
    (2, 255, J, 1, 2, 0.02),     # odd sweep count: result lands in the ping-pong buffer
    (3, 31, RB, 2, 2, 0.004),
    (3, 63, J, 1, 1, 0.001),
    (3, 15, RB, 0, 2, 0.05),     # no pre-smoothing
    (3, 7, RB, 2, 2, 0.3),       # bottom block only
    (2, 3, J, 1, 1, 0.7),        # coarsest grid only: exact solve
    (3, 127, RB, 2, 2, 0.0005),
    (3, 31, J, 0, 1, 0.02),      # no pre-smoothing, Jacobi: coarse levels start from an explicit zero
]


@pytest.mark.parametrize("case", VCYCLE_CASES)
def test_vcycles_match_oracle_fp64(case):
    d, n, sm, nu1, nu2, a = case
    p = O.Problem(d, n, 0.1, 3, 0.05, smoother=sm, nu1=nu1, nu2=nu2)
    rng = np.random.default_rng(n * 7 + d)
    x0 = rng.standard_normal(p.shape)
    b = rng.standard_normal(p.shape)
    ref = x0.copy()
    for _ in range(3):
        ref = O.vcycle(p, a, ref, b)
    g = make_gpu(p)
    x = to_dev(x0)
    g.vcycles(a, x, to_dev(b), 3)
    got = x.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("case", VCYCLE_CASES[:6])
def test_vcycles_fp32_defect_correction(case):
    d, n, sm, nu1, nu2, a = case
    p = O.Problem(d, n, 0.1, 3, 0.05, smoother=sm, nu1=nu1, nu2=nu2)
    rng = np.random.default_rng(n * 11 + d)
    x0, b = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    ref = O.vcycle(p, a, x0, b)
    g = make_gpu(p, vcycle_fp32=True)
    x = to_dev(x0)
    g.vcycles(a, x, to_dev(b), 1)
    got = x.cpu().numpy()
    # one FP32 cycle on the error: FP32 rounding of the correction only
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref - x0).max()


# --- whole time steps (Sec. 2 Eq. 4, Sec. 3) ----------------------------------
STEP_CASES = [
    # ndim, n, nu, M, dt, reaction, smoother, nu1, nu2, L
    (2, 63, 0.1, 3, 0.05, O.REACTION_ALLEN_CAHN, J, 1, 1, 2),
    (3, 31, 0.1, 5, 0.02, O.REACTION_ALLEN_CAHN, RB, 2, 2, 2),
    (2, 31, 0.5, 7, 0.01, O.REACTION_ALLEN_CAHN, RB, 2, 2, 1),
    (3, 15, 0.05, 3, 0.05, O.REACTION_NONE, J, 1, 1, 2),
    (2, 127, 1.0, 2, 0.002, O.REACTION_ALLEN_CAHN, RB, 1, 1, 3),
    (3, 63, 0.3, 3, 0.01, O.REACTION_ALLEN_CAHN, J, 2, 1, 2),
]


@pytest.mark.parametrize("case", STEP_CASES)
def test_steps_match_oracle_fp64(case):
    d, n, nu, M, dt, reaction, sm, nu1, nu2, L = case
    p = O.Problem(d, n, nu, M, dt, reaction=reaction, smoother=sm, nu1=nu1, nu2=nu2, max_sweeps=100)
    u0 = initial_condition(d, n, seed=100 + n + d)
    ref = O.integrate(p, u0, 3, 0, L)
    g = make_gpu(p)
    g.record_history(True)
    u = to_dev(u0)
    for s in range(3):
        g.step(u, ref.sweeps[s], L)
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-12
        hist = g.history()
        # the SDC residual is a difference of O(dt |f|) terms: ~1e-14 absolute rounding floor
        np.testing.assert_allclose(hist, ref.residuals[s], rtol=1e-6, atol=1e-13)


def test_workload_2d_127_ten_steps():
    """The 127^2 workload at full size: 10 steps, sweeps to residual 1e-10."""
    w = workload_2d_127()
    p = O.Problem(2, w.n, w.nu, w.M, w.dt, smoother=J, max_sweeps=100)
    u0 = initial_condition(2, w.n, w.seed)
    ref = O.integrate(p, u0, w.steps, 0, w.n_vcycles)
    assert all(s == 0 for s in ref.status)
    g = make_gpu(p)
    u = to_dev(u0)
    for s in range(w.steps):
        g.step(u, ref.sweeps[s], w.n_vcycles)
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-12
    # the until-tolerance mode reaches the same collocation solution
    u2 = to_dev(u0)
    for s in range(w.steps):
        g.step(u2, 0, w.n_vcycles)
        sweeps, vcyc = g.stats()
        assert abs(sweeps - ref.sweeps[s]) <= 1 and vcyc == sweeps * (w.M - 1) * w.n_vcycles
        assert g.residual() < w.tol
    assert rel_l2(u2.cpu().numpy(), ref.u) <= 1e-9


def test_workload_3d_255_one_sweep_full_size():
    """The 255^3, M=5, V(2,2) red-black Gauss-Seidel workload at full size:
    one sweep element by element against the oracle."""
    w = workload_3d_255()
    p = O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, w.n, w.seed)
    ref = O.isdc_step(p, u0, 1, w.n_vcycles, want_nodes=True)
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, 1, w.n_vcycles)
    nodes = g.nodes().cpu().numpy()
    for m in range(w.M):
        assert rel_l2(nodes[m], ref.nodes[m]) <= 1e-12
    assert abs(g.residual() - ref.residuals[0]) <= 1e-10 * ref.residuals[0]


def test_workload_3d_255_converged_residual_full_size():
    """Full size until the SDC residual is below 1e-10: the oracle recomputes
    the residual of the GPU's node values (a property at any size)."""
    w = workload_3d_255()
    p = O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, w.n, w.seed)
    g = make_gpu(O.Problem(3, w.n, w.nu, w.M, w.dt, smoother=RB, nu1=2, nu2=2, max_sweeps=200))
    u = to_dev(u0)
    st = g.step(u, 0, w.n_vcycles)
    assert st == 0
    R = g.residual()
    assert R < 1e-10
    nodes = g.nodes().cpu().numpy()
    R_oracle = O.sdc_residual(p, nodes)
    assert abs(R_oracle - R) <= 1e-13, (R, R_oracle)
    np.testing.assert_array_equal(nodes[0], u0)
    np.testing.assert_array_equal(nodes[-1], u.cpu().numpy())


# --- mixed precision ----------------------------------------------------------
@pytest.mark.parametrize("case", [(3, 63, 0.1, 5, 0.02, RB, 2, 2), (2, 127, 0.1, 3, 0.05, J, 1, 1),
                                  (3, 31, 0.8, 3, 0.02, J, 1, 1)])
def test_fp32_vcycles_converge_to_fp64_oracle(case):
    d, n, nu, M, dt, sm, nu1, nu2 = case
    p = O.Problem(d, n, nu, M, dt, smoother=sm, nu1=nu1, nu2=nu2, max_sweeps=150)
    u0 = initial_condition(d, n, seed=300 + n)
    ref = O.integrate(p, u0, 2, 0, 2)
    assert all(s == 0 for s in ref.status)
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(u0)
    for s in range(2):
        assert g.step(u, 0, 2) == 0
        assert g.residual() < 1e-10
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-9


@pytest.mark.parametrize("fp32", [False, True])
def test_collocation_solution_is_a_fixed_point_on_gpu(fp32):
    p = O.Problem(3, 15, 0.3, 5, 0.03, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, 15, seed=3)
    pe = O.Problem(3, 15, 0.3, 5, 0.03, solver=O.SOLVER_EXACT, tol=1e-14, max_sweeps=300)
    coll = O.isdc_step(pe, u0, 0, 0, want_nodes=True).nodes
    g = make_gpu(p, vcycle_fp32=fp32)
    g.set_nodes(to_dev(coll))
    u = to_dev(u0)
    g.step(u, 1, 2)
    moved = np.abs(g.nodes().cpu().numpy() - coll).max()
    assert moved <= (1e-11 if fp32 else 1e-13), moved


# --- classical SDC and statuses -------------------------------------------------
def test_classical_sdc_mode_matches_oracle():
    p = O.Problem(2, 63, 1.0, 3, 0.01, reaction=O.REACTION_NONE, smoother=J, solver=O.SOLVER_MG_TOL,
                  mg_tol=1e-9, tol=1e-9)
    u0 = initial_condition(2, 63, seed=8)
    ref = O.isdc_step(p, u0, 0, 0)
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, ref.sweeps, 0)
    sweeps, vcyc = g.stats()
    assert sweeps == ref.sweeps
    assert abs(vcyc - ref.vcycles) <= 2
    assert rel_l2(u.cpu().numpy(), ref.u) <= 1e-9


def test_not_converged_is_soft_and_keeps_last_sweep():
    p = O.Problem(2, 31, 0.1, 3, 0.05, smoother=J, tol=1e-30, max_sweeps=3)
    u0 = initial_condition(2, 31, seed=4)
    ref = O.isdc_step(p, u0, 3, 2)
    g = make_gpu(p)
    u = to_dev(u0)
    import paper_1401_7824_gb300 as G
    assert g.step(u, 0, 2) == G.ISDC_ERR_NOT_CONVERGED
    assert rel_l2(u.cpu().numpy(), ref.u) <= 1e-12


def test_nonfinite_input_reports_status():
    import paper_1401_7824_gb300 as G
    p = O.Problem(2, 31, 0.1, 3, 0.05)
    u0 = initial_condition(2, 31, seed=4)
    u0[5, 5] = np.nan
    g = make_gpu(p)
    with pytest.raises(G.IsdcError) as e:
        g.step(to_dev(u0), 0, 2)
    assert e.value.status == G.ISDC_ERR_NONFINITE


def test_step_host_equals_device_step():
    p = O.Problem(3, 31, 0.1, 5, 0.02, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, 31, seed=12)
    g = make_gpu(p)
    ud = to_dev(u0)
    g.step(ud, 4, 2)
    uh = u0.copy()
    g.step_host(uh, 4, 2)
    np.testing.assert_array_equal(uh, ud.cpu().numpy())


def test_invalid_arguments_are_rejected():
    import paper_1401_7824_gb300 as G
    with pytest.raises(G.IsdcError) as e:
        G.isdc_create(2, 64, 0.1, 3, 0.05)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
    with pytest.raises(G.IsdcError) as e:
        G.isdc_create(2, 63, 0.1, 3, 0.05, nodes=7)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
    with pytest.raises(G.IsdcError) as e:
        G.isdc_create(3, 31, -1.0, 3, 0.05)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("dim,n,sm", [(3, 31, RB), (3, 127, RB), (2, 255, J)])
def test_sweep_graph_replay_is_bitwise_identical(fp32, dim, n, sm):
    """A sweep replayed from its captured CUDA graph (with programmatic
    dependencies between kernels, the default, and with ordinary ones) runs the
    same kernels in the same order as launching them one by one: the same
    values bit for bit, so every kernel's entry wait orders it after the one
    before it."""
    p = O.Problem(dim, n, 0.1, 5, 0.02, smoother=sm, nu1=2, nu2=2, max_sweeps=150)
    u0 = initial_condition(dim, n, seed=21)
    outs = []
    for graphs in (1, 2, 0):
        g = make_gpu(p, vcycle_fp32=fp32, use_graphs=graphs, fused_transfer=0, rb_run=4 if dim == 3 else 0)
        u = to_dev(u0)
        for _ in range(2):
            g.step(u, 0, 2)
        outs.append((u.cpu().numpy(), g.stats(), g.history()))
        g.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0][0], o[0])
        assert outs[0][1] == o[1]
        assert outs[0][2] == o[2]


def test_fp32_red_black_2d_split_layout_converges_to_oracle():
    """2D red-black smoothing with FP32 V-cycles uses the colour-split fine level."""
    p = O.Problem(2, 255, 0.2, 5, 0.02, smoother=RB, nu1=2, nu2=2, max_sweeps=150)
    u0 = initial_condition(2, 255, seed=17)
    ref = O.integrate(p, u0, 2, 0, 2)
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(u0)
    for s in range(2):
        assert g.step(u, 0, 2) == 0
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-9


def test_largest_grid_allocates_and_a_second_reports_oom():
    """The largest grid (3D side 1023, M = 7: ~200 GB of node state and
    hierarchy) allocates; a second one does not fit beside it and fails cleanly
    with ISDC_ERR_OOM (an allocation failure; nothing is launched)."""
    import paper_1401_7824_gb300 as G
    big = G.isdc_create(3, 1023, 0.1, 7, 0.01)
    try:
        with pytest.raises(G.IsdcError) as e:
            G.isdc_create(3, 1023, 0.1, 7, 0.01)
        assert e.value.status == G.ISDC_ERR_OOM
    finally:
        G.isdc_destroy(big)
    g = make_gpu(O.Problem(2, 63, 0.1, 3, 0.05))  # the device is still usable afterwards
    u = to_dev(initial_condition(2, 63, seed=1))
    assert g.step(u, 2, 2) == 0


def test_mid_step_checkpoint_resumes_bitwise():
    """Checkpoint / resume: node values saved after 3 sweeps and restored in a
    fresh context continue exactly like an uninterrupted 5-sweep step (a sweep
    depends only on the node values and f of the previous one)."""
    p = O.Problem(3, 31, 0.1, 5, 0.02, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, 31, seed=23)
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, 5, 2)
    g2 = make_gpu(p)
    v = to_dev(u0)
    g2.step(v, 3, 2)
    ckpt = g2.nodes().clone()
    g3 = make_gpu(p)
    g3.set_nodes(ckpt)
    w = to_dev(u0)
    g3.step(w, 2, 2)
    np.testing.assert_array_equal(w.cpu().numpy(), u.cpu().numpy())
    np.testing.assert_array_equal(g3.nodes().cpu().numpy(), g.nodes().cpu().numpy())


@pytest.mark.parametrize("nu12", [(2, 2), (3, 1)])
def test_temporal_blocking_is_bitwise_identical(nu12):
    """Blocked passes of 1 or 2 red-black sweeps over the FP32 colour-split fine
    level (3D) do the same FP32 operations in the same order as one pass per
    colour, so whole steps agree bit for bit; the result still matches the
    oracle.  Side 127: several tiles in x and y, several z-chunks, ragged edges."""
    import paper_1401_7824_gb300 as G
    nu1, nu2 = nu12
    p = O.Problem(3, 127, 0.1, 3, 0.02, smoother=RB, nu1=nu1, nu2=nu2, max_sweeps=150)
    u0 = initial_condition(3, 127, seed=41)
    outs = []
    for depth in (0, 1, 2):
        g = make_gpu(p, vcycle_fp32=True, temporal_blocking=depth)
        assert g.tuning()["tb_depth"] == depth
        u = to_dev(u0)
        assert g.step(u, 0, 2) == 0
        outs.append((u.cpu().numpy(), g.stats(), g.residual()))
        g.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        assert o[1] == outs[0][1] and o[2] == outs[0][2]
    ref = O.integrate(p, u0, 1, 0, 2)
    assert rel_l2(outs[0][0], ref.per_step_u[0]) <= 1e-9


@pytest.mark.parametrize("fp32", [False, True])
def test_red_black_run_forms_are_bitwise_identical(fp32):
    """The 3D red-black colour pass of the natural-layout levels walks diagonal
    runs and shares pair sums between consecutive points; every run length and
    both issue orders (streamed, or all loads first) form each point's sum as
    (x-pair + lower pair) + upper pair, so whole steps agree bit for bit.  FP64
    V-cycles on side 63 (levels 63, 31, 15 in the pass: ragged runs at the
    grid's edges, several blocks along every axis; checked against the oracle
    too) and FP32 V-cycles on side 127 (coarse levels 63 and 31 in the pass)."""
    n = 127 if fp32 else 63
    p = O.Problem(3, n, 0.1, 3, 0.02, smoother=RB, nu1=2, nu2=2, max_sweeps=150)
    u0 = initial_condition(3, n, seed=43)
    outs = []
    for run in (1, 2, 4, 8, 16, 32, -1, -2, -4, -8):
        g = make_gpu(p, vcycle_fp32=fp32, rb_run=run)
        if not fp32:
            assert g.tuning()["zb_fp64"] == abs(run)
        u = to_dev(u0)
        assert g.step(u, 0, 2) == 0
        outs.append((u.cpu().numpy(), g.stats(), g.residual()))
        g.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        assert o[1] == outs[0][1] and o[2] == outs[0][2]
    if not fp32:
        ref = O.integrate(p, u0, 1, 0, 2)
        assert rel_l2(outs[0][0], ref.per_step_u[0]) <= 1e-12


FUSED_CASES = [
    # ndim, n, smoother, nu1, nu2, fp32 V-cycles
    (3, 255, RB, 2, 2, False),   # red-only residual; coarse sides 127, 63, 31, 15 ragged against 32 x 8 tiles
    (3, 127, J, 1, 1, False),    # full residual (27-term full weighting)
    (3, 255, RB, 2, 2, True),    # colour-split FP32 fine level, then natural FP32 levels
    (3, 63, J, 1, 2, True),
    (2, 1023, RB, 1, 1, False),  # 2D tiles, red-only
    (2, 511, J, 1, 1, False),
    (2, 1023, RB, 2, 2, True),
    (2, 255, J, 1, 1, True),
]


@pytest.mark.parametrize("case", FUSED_CASES)
def test_fused_residual_restriction_is_bitwise_identical(case):
    """Residual + full weighting in one launch (the residual kept in shared
    memory, tiles of 32 x 8 coarse points walking z) against the two-launch form
    (the residual written to device memory and read back): the same expressions
    in the same order, so three V-cycles agree bit for bit; the FP64 cases are
    also checked against the oracle's V-cycles."""
    d, n, sm, nu1, nu2, fp32 = case
    p = O.Problem(d, n, 0.1, 3, 0.02, smoother=sm, nu1=nu1, nu2=nu2)
    rng = np.random.default_rng(n * 13 + d)
    x0, b = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    a = 0.02 if d == 2 else 0.004
    outs = []
    for fused in (True, False):
        g = make_gpu(p, vcycle_fp32=fp32, fused_transfer=fused)
        x = to_dev(x0)
        g.vcycles(a, x, to_dev(b), 3)
        outs.append(x.cpu().numpy())
        g.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    if not fp32:
        ref = x0.copy()
        for _ in range(3):
            ref = O.vcycle(p, a, ref, b)
        assert np.abs(outs[0] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fused_transfer_whole_steps_match_two_launch_form():
    """Whole until-tolerance steps of the 127^3 FP32-V-cycle workload with the
    fused and the two-launch transfer agree bit for bit (values, sweep counts
    and residuals)."""
    n = 127
    p = O.Problem(3, n, 0.1, 5, 0.02, smoother=RB, nu1=2, nu2=2, max_sweeps=150)
    u0 = initial_condition(3, n, seed=44)
    outs = []
    for fused in (True, False):
        g = make_gpu(p, vcycle_fp32=True, fused_transfer=fused)
        u = to_dev(u0)
        assert g.step(u, 0, 2) == 0
        outs.append((u.cpu().numpy(), g.stats(), g.residual()))
        g.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]
    g = make_gpu(p, vcycle_fp32=True)  # default: each level's form chosen by the autotuner
    kc = g.tuning()["transfer_kc"]
    assert len(kc) >= 2 and all(k in (0, 4, 8, 16) for k in kc), kc
    u = to_dev(u0)
    assert g.step(u, 0, 2) == 0
    np.testing.assert_array_equal(u.cpu().numpy(), outs[0][0])
    g.close()


def test_transfer_tuner_skips_fused_form_on_underfilled_levels():
    """The fused residual + restriction is offered to the autotuner only on
    levels whose fused grid has at least two blocks per SM: on the 127^2
    workload (coarse sides 63 and below) every level keeps the two launches."""
    p = O.Problem(2, 127, 0.1, 3, 0.05)
    g = make_gpu(p)
    kc = g.tuning()["transfer_kc"]
    g.close()
    assert len(kc) >= 1 and all(k == 0 for k in kc), kc


def test_red_black_run_option_is_validated():
    import paper_1401_7824_gb300 as G
    p = O.Problem(3, 31, 0.1, 3, 0.02, smoother=RB, nu1=2, nu2=2)
    for bad in (3, -16, 64):
        with pytest.raises(G.IsdcError) as e:
            make_gpu(p, rb_run=bad)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG


def test_temporal_blocking_option_is_validated_and_tuned():
    import paper_1401_7824_gb300 as G
    p = O.Problem(3, 63, 0.1, 3, 0.02, smoother=RB, nu1=2, nu2=2)
    g = make_gpu(p, vcycle_fp32=True)
    t = g.tuning()
    assert t["tb_depth"] in (0, 1, 2) and t["tb_planes"] in (16, 32, 64, 128)
    g.close()
    with pytest.raises(G.IsdcError) as e:
        make_gpu(p, vcycle_fp32=True, temporal_blocking=3)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG



# --- Gauss-Radau (right) and Gauss-Legendre nodes (Sec. 2) ---------------------
RL = (O.NODES_RADAU_RIGHT, O.NODES_LEGENDRE)
NODE_STEP_CASES = [
    # ndim, n, nu, M, dt, smoother, nu1, nu2, L, nodes
    (2, 63, 0.1, 3, 0.05, J, 1, 1, 2, O.NODES_RADAU_RIGHT),
    (2, 63, 0.1, 3, 0.05, J, 1, 1, 2, O.NODES_LEGENDRE),
    (3, 31, 0.1, 5, 0.02, RB, 2, 2, 2, O.NODES_RADAU_RIGHT),
    (3, 31, 0.1, 4, 0.02, RB, 2, 2, 2, O.NODES_LEGENDRE),
    (2, 31, 0.5, 7, 0.01, RB, 2, 2, 1, O.NODES_LEGENDRE),
    (3, 15, 0.3, 2, 0.05, J, 1, 1, 3, O.NODES_RADAU_RIGHT),
]


@pytest.mark.parametrize("case", NODE_STEP_CASES)
def test_radau_legendre_steps_match_oracle_fp64(case):
    """M node solves per sweep from t_0; Gauss-Legendre ends each step with the
    full-step quadrature.  FP64 path against the oracle, relative L2 <= 1e-12."""
    d, n, nu, M, dt, sm, nu1, nu2, L, kind = case
    p = O.Problem(d, n, nu, M, dt, smoother=sm, nu1=nu1, nu2=nu2, max_sweeps=100, nodes=kind)
    u0 = initial_condition(d, n, seed=400 + n + d + M)
    ref = O.integrate(p, u0, 3, 0, L)
    assert all(st == 0 for st in ref.status)
    g = make_gpu(p)
    g.record_history(True)
    u = to_dev(u0)
    for s in range(3):
        g.step(u, ref.sweeps[s], L)
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-12
        np.testing.assert_allclose(g.history(), ref.residuals[s], rtol=1e-6, atol=1e-13)
        sweeps, vcyc = g.stats()
        assert vcyc == sweeps * M * L


@pytest.mark.parametrize("kind", RL)
def test_radau_legendre_fp32_vcycles_converge_to_oracle(kind):
    p = O.Problem(3, 63, 0.1, 3, 0.02, smoother=RB, nu1=2, nu2=2, max_sweeps=150, nodes=kind)
    u0 = initial_condition(3, 63, seed=430 + kind)
    ref = O.integrate(p, u0, 2, 0, 2)
    g = make_gpu(p, vcycle_fp32=True)
    u = to_dev(u0)
    for s in range(2):
        assert g.step(u, 0, 2) == 0
        assert g.residual() < 1e-10
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-9


@pytest.mark.parametrize("kind", RL)
def test_radau_legendre_nodes_residual_and_resume(kind):
    """Node values come back without t_0; the oracle's residual of them (with
    u_0 given) equals the library's; resuming from them is bitwise."""
    p = O.Problem(2, 63, 0.2, 3, 0.03, smoother=J, nodes=kind)
    u0 = initial_condition(2, 63, seed=440 + kind)
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, 5, 2)
    nodes = g.nodes().cpu().numpy()
    assert nodes.shape == (3,) + p.shape
    assert abs(O.sdc_residual(p, nodes, u0) - g.residual()) <= 1e-13
    g2 = make_gpu(p)
    v = to_dev(u0)
    g2.step(v, 3, 2)
    g3 = make_gpu(p)
    g3.set_nodes(g2.nodes().clone())
    w = to_dev(u0)
    g3.step(w, 2, 2)
    np.testing.assert_array_equal(w.cpu().numpy(), u.cpu().numpy())


@pytest.mark.parametrize("kind", RL)
def test_radau_legendre_graph_replay_is_bitwise_identical(kind):
    p = O.Problem(3, 31, 0.1, 3, 0.02, smoother=RB, nu1=2, nu2=2, nodes=kind)
    u0 = initial_condition(3, 31, seed=450 + kind)
    outs = []
    for graphs in (True, False):
        g = make_gpu(p, vcycle_fp32=True, use_graphs=graphs)
        u = to_dev(u0)
        g.step(u, 0, 2)
        outs.append((u.cpu().numpy(), g.stats()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_profiler_counts_only_and_event_modes_agree():
    """Counting without events (no per-sweep synchronisation) and timing one
    class with events give the same launch counts, bytes and ops per class for
    the same work; only the timed class gets a duration (-1 marks an untimed
    class); results do not change."""
    p = O.Problem(3, 31, 0.1, 5, 0.02, smoother=RB, nu1=2, nu2=2)
    u0 = initial_condition(3, 31, seed=25)
    reads, outs = [], []
    for classes in ([], ["smooth_fine"], None):
        g = make_gpu(p)
        u = to_dev(u0)
        g.step(u, 2, 2)
        if classes is None:
            g.step(u, 3, 2)
        else:
            g.profile(True, classes=classes)
            g.step(u, 3, 2)
            reads.append(g.profile_read())
            g.profile(False)
        outs.append(u.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[1], outs[2])
    a, b = reads
    assert a.keys() == b.keys() and "smooth_fine" in a
    for k in a:
        assert a[k]["launches"] == b[k]["launches"] and a[k]["bytes"] == b[k]["bytes"]
        assert a[k]["total_ms"] == -1.0                         # not timed
        assert (b[k]["total_ms"] > 0.0) == (k == "smooth_fine")  # only the named class is timed
