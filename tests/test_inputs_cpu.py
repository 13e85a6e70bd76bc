"""The seeded input recipes (isdc_inputs.py) match the recipe the design notes
state: grid convention, initial data, the workload parameters, and the batch
and request streams.  CPU only; these generators feed the oracle, the CUDA
parity tests and the benchmark alike."""
import numpy as np

import isdc_inputs as W


def test_grid_convention_and_sine_mode():
    n = 7
    x = W.grid_coords(n)
    np.testing.assert_allclose(x, np.arange(1, 8) / 8.0, rtol=0, atol=0)
    u2 = W.sine_mode(2, n)
    assert u2.shape == (n, n) and u2.flags["C_CONTIGUOUS"]
    # x fastest: varying the last index moves along x
    u = W.sine_mode(2, n, p=(1, 2))
    np.testing.assert_allclose(u[3, :], np.sin(np.pi * x) * np.sin(2 * np.pi * x[3]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(u[:, 3], np.sin(np.pi * x[3]) * np.sin(2 * np.pi * x), rtol=0, atol=1e-15)
    u3 = W.sine_mode(3, n, p=(1, 2, 3))
    assert u3.shape == (n, n, n)
    np.testing.assert_allclose(u3[2, 4, :], np.sin(np.pi * x) * np.sin(2 * np.pi * x[4]) * np.sin(3 * np.pi * x[2]),
                               rtol=0, atol=1e-15)


def test_initial_condition_is_sine_product_plus_seeded_noise():
    a = W.initial_condition(2, 127, seed=1)
    b = W.initial_condition(2, 127, seed=1)
    c = W.initial_condition(2, 127, seed=2)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    noise = a - W.sine_mode(2, 127)
    assert abs(noise.mean()) < 3 * 0.01 / 127          # N(0, 0.01^2): mean within 3 standard errors
    assert abs(noise.std() / 0.01 - 1.0) < 0.03         # 16 129 draws: std within 3 %
    np.testing.assert_array_equal(W.initial_condition(2, 31, seed=5, noise_std=0.0), W.sine_mode(2, 31))


def test_workload_parameters():
    w = W.workload_2d_127()
    assert (w.ndim, w.n, w.nu, w.M, w.dt, w.steps, w.n_vcycles, w.smoother, w.nu1, w.nu2, w.seed) == \
        (2, 127, 0.1, 3, 0.05, 10, 2, 0, 1, 1, 1)
    w = W.workload_3d_255()
    assert (w.ndim, w.n, w.nu, w.M, w.dt, w.steps, w.n_vcycles, w.smoother, w.nu1, w.nu2, w.seed) == \
        (3, 255, 0.1, 5, 0.02, 20, 2, 1, 2, 2, 2)
    assert w.N == 16_581_375 and w.reaction == 1 and not w.vcycle_fp32
    w = W.workload_3d_511_mixed()
    assert (w.ndim, w.n, w.M, w.dt, w.vcycle_fp32, w.seed) == (3, 511, 5, 0.02, True, 3)
    assert 0.01 <= w.nu <= 1.0 and abs(w.nu - 0.0148) < 5e-5  # nu = 10^U(-2, 0) from seed 3
    assert W.workload_3d_255_radau().nodes == 1 and W.workload_3d_255_legendre().nodes == 2
    w = W.workload_2d_1023_compact()
    assert (w.ndim, w.n, w.stencil, w.smoother) == (2, 1023, 1, 0)
    w = W.workload_2d_1024_burgers()
    assert (w.ndim, w.n, w.equation, w.reaction, w.smoother) == (2, 1024, 1, 0, 1)


def test_workload_initial_dispatch_and_periodic_bump():
    w = W.workload_2d_1024_burgers()
    n = 64
    u = W.periodic_bump(2, n, seed=w.seed, noise_std=0.0)
    x = W.periodic_grid_coords(n)
    assert x[0] == -1.0 and x[n // 2] == 0.0 and abs(x[-1] - (1.0 - 2.0 / n)) < 1e-15
    assert u[n // 2, n // 2] == 1.0 and u.max() == 1.0
    np.testing.assert_allclose(u[n // 2, :], np.exp(-x ** 2 / 0.01), rtol=0, atol=1e-15)
    small = W.Workload("t", 2, n, 0.1, 3, 0.01, 1, 2, 1, 2, 2, reaction=0, seed=7, equation=1)
    np.testing.assert_array_equal(W.workload_initial(small), W.periodic_bump(2, n, 7))
    heat = W.Workload("t", 2, 31, 0.1, 3, 0.01, 1, 2, 0, 1, 1, seed=3)
    np.testing.assert_array_equal(W.workload_initial(heat), W.initial_condition(2, 31, 3))


def test_batch_instances_3d_recipe():
    """The 3D batch: 32 instances with the 3D request mix's sides (2^j - 1,
    j in 6..8), red-black V(2,2) settings, seeded and reproducible."""
    inst = W.batch_instances_3d()
    assert len(inst) == 32
    assert {w.n for w in inst} == {63, 127, 255}
    for w in inst:
        assert w.ndim == 3 and w.M in (3, 5) and 0.01 <= w.nu <= 1.0 and 0.01 <= w.dt <= 0.1
        assert (w.smoother, w.nu1, w.nu2, w.n_vcycles) == (1, 2, 2, 2) and w.vcycle_fp32
    assert len({w.seed for w in inst}) == 32
    again = W.batch_instances_3d()
    assert [(w.n, w.nu, w.M, w.dt, w.seed) for w in inst] == [(w.n, w.nu, w.M, w.dt, w.seed) for w in again]
    assert sum(w.n ** 3 for w in inst) == 167_425_504  # the bench line's dofs_total


def test_batch_instances_recipe():
    inst = W.batch_instances()
    assert len(inst) == 256
    sides = {w.n for w in inst}
    assert sides <= {63, 127, 255, 511, 1023} and len(sides) == 5
    for w in inst:
        assert w.ndim == 2 and w.M in (3, 5) and 0.01 <= w.nu <= 1.0 and 0.01 <= w.dt <= 0.1
        assert (w.smoother, w.nu1, w.nu2, w.n_vcycles) == (0, 1, 1, 2) and w.vcycle_fp32
    # the expected points per instance of a uniform j in 6..10 (2D): 278 554.6
    assert abs(np.mean([(2 ** j - 1) ** 2 for j in range(6, 11)]) - 278_554.6) < 1e-6
    again = W.batch_instances()
    assert [(w.n, w.nu, w.dt, w.M) for w in inst] == [(w.n, w.nu, w.dt, w.M) for w in again]


def test_request_stream_recipe():
    reqs = W.request_stream()
    assert len(reqs) == 2000
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.1            # Poisson arrivals at 200 per second
    frac2d = np.mean([w.ndim == 2 for _, w in reqs])
    assert abs(frac2d - 0.7) < 0.05
    for _, w in reqs:
        if w.ndim == 2:
            assert w.n in (127, 255, 511, 1023) and (w.smoother, w.nu1, w.nu2) == (0, 1, 1)
        else:
            assert w.n in (63, 127, 255) and (w.smoother, w.nu1, w.nu2) == (1, 2, 2)
        assert w.M in (3, 5) and w.steps == 10
