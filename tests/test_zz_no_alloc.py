"""The allocation-free V-cycle entry point, isdc_vcycles_static.

It serves callers that cannot allocate device memory (code under another
framework's memory manager, real-time loops, code that must not allocate
during graph capture): its multigrid buffers live in a static device array.
These tests call it through the C ABI and check it against the context-based
isdc_vcycles and against the oracle's V-cycles on the same inputs, on two
calls in a row, within the FP64 V-cycle tolerance used elsewhere (1e-12
relative to the solution size)."""
import numpy as np
import pytest

import oracle as O
from gpu_util import make_gpu, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # ndim, n, smoother, nu1, nu2, a
    (2, 1023, O.SMOOTHER_JACOBI, 1, 1, 0.002),   # largest 2D side that fits the static array
    (3, 127, O.SMOOTHER_JACOBI, 1, 1, 0.0005),   # largest 3D side that fits
    (3, 63, O.SMOOTHER_RBGS, 2, 2, 0.004),
    (2, 31, O.SMOOTHER_RBGS, 1, 2, 0.05),        # bottom block only
]


@pytest.mark.parametrize("case", CASES)
def test_static_vcycles_match_context_vcycles_twice(case):
    import paper_1401_7824_gb300 as G
    d, n, sm, nu1, nu2, a = case
    p = O.Problem(d, n, 0.1, 3, 0.05, smoother=sm, nu1=nu1, nu2=nu2)
    g = make_gpu(p)
    rng = np.random.default_rng(1000 + n)
    x0 = rng.standard_normal(p.shape)
    bs = [rng.standard_normal(p.shape), rng.standard_normal(p.shape)]
    a_s = [a, 1.7 * a]
    x_ctx, x_static = to_dev(x0), to_dev(x0)
    x_orc = x0.copy()
    for call in range(2):  # the second call reuses the static array left by the first
        b = to_dev(bs[call])
        g.vcycles(a_s[call], x_ctx, b, 2)
        G.isdc_vcycles_static(d, n, a_s[call], x_static, b, 2, smoother=sm, nu1=nu1, nu2=nu2, omega=p.omega)
        for _ in range(2):
            x_orc = O.vcycle(p, a_s[call], x_orc, bs[call])
        ref = x_ctx.cpu().numpy()
        got = x_static.cpu().numpy()
        scale = np.abs(x_orc).max()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), call
        assert np.abs(got - x_orc).max() <= 1e-12 * scale, call  # and the FP64 oracle's V-cycles
    g.close()


def test_static_vcycles_take_no_device_memory():
    """After a first call per smoother (which looks up the static array's
    address and loads the kernels), further calls leave the device's free memory unchanged: the entry point allocates
    nothing, and torch's caching allocator is not touched between the reads."""
    import paper_1401_7824_gb300 as G
    torch = pytest.importorskip("torch")
    n = 255
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    b = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    for sm in (G.ISDC_SMOOTHER_JACOBI, G.ISDC_SMOOTHER_RBGS):  # kernels loaded lazily on first use
        G.isdc_vcycles_static(2, n, 0.01, x, b, 1, smoother=sm)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for sm in (G.ISDC_SMOOTHER_JACOBI, G.ISDC_SMOOTHER_RBGS):
        for _ in range(3):
            G.isdc_vcycles_static(2, n, 0.01, x, b, 2, smoother=sm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.isfinite(x).all()


def test_static_vcycles_reject_grids_beyond_the_array():
    import paper_1401_7824_gb300 as G
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    for d, n in [(3, 255), (2, 2047)]:
        with pytest.raises(G.IsdcError) as e:
            G.isdc_vcycles_static(d, n, 0.01, x, x, 1)
        assert e.value.status == G.ISDC_ERR_SCRATCH_TOO_SMALL
