"""The all-core oracle build (the same C file compiled with -fopenmp; only the
outermost grid loops are split over threads, max-norms combine per-thread
maxima) gives the plain build's results bit for bit: V-cycles with both
smoothers, exact sine-transform solves, whole until-tolerance ISDC steps and
the SDC residual, in 2D and 3D, on ragged sizes."""
import numpy as np
import pytest

import oracle as O
from isdc_inputs import initial_condition


@pytest.fixture(scope="module", autouse=True)
def four_threads():
    O.set_threads(4)
    with O.all_cores():
        assert O.threads() == 4
    assert O.threads() == 1
    yield


def _both(fn):
    plain = fn()
    with O.all_cores():
        threaded = fn()
    return plain, threaded


@pytest.mark.parametrize("d,n,sm", [(2, 63, O.SMOOTHER_JACOBI), (2, 127, O.SMOOTHER_RBGS),
                                    (3, 15, O.SMOOTHER_RBGS), (3, 31, O.SMOOTHER_JACOBI)])
def test_threaded_vcycle_and_exact_solve_bitwise(d, n, sm):
    p = O.Problem(d, n, 0.1, 3, 0.02, smoother=sm, nu1=2, nu2=1)
    rng = np.random.default_rng(5 + n)
    x0, b = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    a, c = _both(lambda: O.vcycle(p, 0.01, O.vcycle(p, 0.01, x0, b), b))
    np.testing.assert_array_equal(a, c)
    a, c = _both(lambda: O.solve_exact(0.01, b))
    np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("d,n,M,sm", [(2, 31, 3, O.SMOOTHER_JACOBI), (3, 15, 5, O.SMOOTHER_RBGS)])
def test_threaded_isdc_step_bitwise(d, n, M, sm):
    p = O.Problem(d, n, 0.1, M, 0.02, smoother=sm, nu1=2, nu2=2)
    u0 = initial_condition(d, n, seed=3)
    a, c = _both(lambda: O.isdc_step(p, u0, 0, 2, want_nodes=True))
    np.testing.assert_array_equal(a.u, c.u)
    np.testing.assert_array_equal(a.nodes, c.nodes)
    assert a.sweeps == c.sweeps and a.vcycles == c.vcycles
    np.testing.assert_array_equal(a.residuals, c.residuals)
    r1, r2 = _both(lambda: O.sdc_residual(p, a.nodes))
    assert r1 == r2
