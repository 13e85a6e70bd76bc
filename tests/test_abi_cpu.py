"""Host-side checks of the C ABI library (no GPU): it builds, loads, exports
every entry point declared in include/isdc.h, and its host-only functions
(collocation tables, argument validation) behave."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(isdc_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import paper_1401_7824_gb300 as G
    lib = G.load()
    declared = _declared()
    assert "isdc_create" in declared and "isdc_step" in declared and "isdc_residual" in declared
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", G.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (isdc_\w+)", out))
    assert exported == set(declared), exported ^ set(declared)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7])
def test_library_collocation_tables_match_oracle(M):
    import paper_1401_7824_gb300 as G
    tau, Q, S = G.isdc_collocation_tables(M)
    np.testing.assert_allclose(tau, O.lobatto_nodes(M), atol=2e-16)
    np.testing.assert_allclose(Q, O.q_matrix(M), atol=2e-15)
    np.testing.assert_allclose(S, O.s_matrix(M), atol=2e-15)


def test_host_validation_without_gpu():
    import paper_1401_7824_gb300 as G
    with pytest.raises(G.IsdcError) as e:
        G.isdc_collocation_tables(3, nodes=G.ISDC_NODES_GAUSS_LEGENDRE)
    assert e.value.status == G.ISDC_ERR_UNSUPPORTED
    with pytest.raises(G.IsdcError) as e:
        G.isdc_collocation_tables(9)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
    for bad in [dict(ndim=4, n=7), dict(ndim=2, n=8), dict(ndim=2, n=1)]:
        with pytest.raises(G.IsdcError) as e:
            G.isdc_create(bad["ndim"], bad["n"], 0.1, 3, 0.05)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG
        assert "must" in G.isdc_last_error()
    o = G.isdc_default_options()
    assert (o.smoother, o.nu1, o.nu2, o.max_sweeps, o.tol) == (0, 1, 1, 100, 1e-10)
