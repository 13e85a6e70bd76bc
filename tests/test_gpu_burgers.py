"""Parity of the CUDA path for the viscous Burgers equation of Sec. 4.1
(periodic grid, WENO5 advection explicit, Laplacian implicit by periodic
multigrid; FP64) against the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
from gpu_util import make_gpu, rel_l2, to_dev

pytestmark = pytest.mark.gpu

B, J, RB = O.EQUATION_BURGERS, O.SMOOTHER_JACOBI, O.SMOOTHER_RBGS


def bump(d, n, seed, sigma=0.25):
    """A periodic Gaussian bump plus seeded N(0, 0.01^2) noise (x fastest)."""
    x = -1.0 + (2.0 / n) * np.arange(n)
    g = np.meshgrid(*([x] * d), indexing="ij")[::-1]
    r2 = sum(c ** 2 for c in g)
    return np.exp(-r2 / sigma ** 2) + 0.01 * np.random.default_rng(seed).standard_normal((n,) * d)


@pytest.mark.parametrize("d,n,sm,nu1,nu2,a", [(2, 64, RB, 2, 2, 0.002), (2, 128, J, 1, 1, 0.0005),
                                               (3, 16, RB, 2, 2, 0.01), (2, 8, J, 1, 2, 0.1)])
def test_periodic_vcycles_match_oracle(d, n, sm, nu1, nu2, a):
    p = O.Problem(d, n, 0.1, 3, 0.01, equation=B, smoother=sm, nu1=nu1, nu2=nu2)
    rng = np.random.default_rng(600 + n + d)
    x0, b = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    ref = x0.copy()
    for _ in range(3):
        ref = O.vcycle(p, a, ref, b)
    g = make_gpu(p)
    x = to_dev(x0)
    g.vcycles(a, x, to_dev(b), 3)
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


CASES = [
    # d, n, nu, M, dt, smoother, nu1, nu2, L, nodes
    (2, 64, 0.1, 3, 0.002, RB, 2, 2, 2, O.NODES_LOBATTO),
    (2, 128, 1.0, 5, 0.001, J, 1, 1, 2, O.NODES_LOBATTO),
    (2, 32, 0.05, 3, 0.005, RB, 2, 2, 2, O.NODES_RADAU_RIGHT),
    (2, 32, 0.5, 2, 0.004, J, 2, 2, 3, O.NODES_LEGENDRE),
    (3, 16, 0.2, 3, 0.004, RB, 2, 2, 2, O.NODES_LOBATTO),
]


@pytest.mark.parametrize("case", CASES)
def test_burgers_steps_match_oracle(case):
    d, n, nu, M, dt, sm, nu1, nu2, L, kind = case
    p = O.Problem(d, n, nu, M, dt, equation=B, smoother=sm, nu1=nu1, nu2=nu2, max_sweeps=100, nodes=kind)
    u0 = bump(d, n, seed=610 + n)
    ref = O.integrate(p, u0, 3, 0, L)
    assert all(st == 0 for st in ref.status)
    g = make_gpu(p)
    g.record_history(True)
    u = to_dev(u0)
    for s in range(3):
        g.step(u, ref.sweeps[s], L)
        assert rel_l2(u.cpu().numpy(), ref.per_step_u[s]) <= 1e-12
        np.testing.assert_allclose(g.history(), ref.residuals[s], rtol=1e-6, atol=1e-13)


def test_burgers_until_tolerance_graph_and_resume():
    p = O.Problem(2, 64, 0.3, 3, 0.002, equation=B, smoother=RB, nu1=2, nu2=2, max_sweeps=100)
    u0 = bump(2, 64, seed=620)
    ref = O.isdc_step(p, u0, 0, 2)
    outs = []
    for graphs in (True, False):
        g = make_gpu(p, use_graphs=graphs)
        u = to_dev(u0)
        assert g.step(u, 0, 2) == 0
        outs.append((u.cpu().numpy(), g.stats()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    assert abs(outs[0][1][0] - ref.sweeps) <= 1
    assert rel_l2(outs[0][0], ref.u) <= 1e-9
    g = make_gpu(p)
    u = to_dev(u0)
    g.step(u, 5, 2)
    g2 = make_gpu(p)
    v = to_dev(u0)
    g2.step(v, 3, 2)
    g3 = make_gpu(p)
    g3.set_nodes(g2.nodes().clone())
    w = to_dev(u0)
    g3.step(w, 2, 2)
    np.testing.assert_array_equal(w.cpu().numpy(), u.cpu().numpy())


@pytest.mark.parametrize("nu", [0.1, 1, 10])
@pytest.mark.parametrize("M", [3, 5, 7])
def test_burgers_table1b_counts_match_oracle(nu, M):
    """Table 1b setting (128^2 periodic points, dt = 0.001, residual 5e-8):
    classical SDC (multigrid to 5e-9) and ISDC (L = 2 as a cap) sweep and
    V-cycle counts of the CUDA path against the oracle's."""
    from oracle.table1 import burgers_initial, burgers_problem
    u0 = burgers_initial(128)
    ps, pi = burgers_problem(nu, M, O.SOLVER_MG_TOL), burgers_problem(nu, M, O.SOLVER_ISDC_CAPPED)
    sdc, isdc = O.isdc_step(ps, u0, 0, 0), O.isdc_step(pi, u0, 0, 2)
    g = make_gpu(ps)
    u = to_dev(u0)
    g.step(u, 0, 0)
    gs = g.stats()
    gi = make_gpu(pi, vcycle_cap=True)
    v = to_dev(u0)
    gi.step(v, 0, 2)
    gis = gi.stats()
    assert gs[0] == sdc.sweeps and abs(gs[1] - sdc.vcycles) <= 1
    assert gis[0] == isdc.sweeps and abs(gis[1] - isdc.vcycles) <= 1


def test_burgers_invalid_and_unsupported():
    import paper_1401_7824_gb300 as G
    with pytest.raises(G.IsdcError) as e:
        G.Isdc(2, 63, 0.1, 3, 0.01, equation=G.ISDC_EQUATION_BURGERS)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
    with pytest.raises(G.IsdcError) as e:
        G.Isdc(2, 64, 0.1, 3, 0.01)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
    with pytest.raises(G.IsdcError) as e:
        G.Isdc(2, 64, 0.1, 3, 0.01, equation=G.ISDC_EQUATION_BURGERS, vcycle_fp32=True)
    assert e.value.status == G.ISDC_ERR_UNSUPPORTED
