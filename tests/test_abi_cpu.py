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


def _declared(header="isdc.h"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(isdc_\w+)\s*\(", txt)))


def test_every_header_is_covered():
    assert sorted(h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")) == \
        ["isdc.h", "isdc_probe.h"]


def test_probe_library_exports_its_header():
    import paper_1401_7824_gb300.build as B
    path = B.build_probe()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(re.findall(r" T (isdc_\w+)", out)) == set(_declared("isdc_probe.h")) == {"isdc_probe_fp64_rate"}


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


@pytest.mark.parametrize("kind", ["radau", "legendre"])
@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7])
def test_library_radau_legendre_tables_match_oracle(kind, M):
    """The library's Golub-Welsch nodes and exact Lagrange integrals against the
    oracle's (root bracketing / Newton, Gauss quadrature of l_j); S runs over the
    M steps t_0 -> t_1 -> ... -> t_M (Eq. 2)."""
    import paper_1401_7824_gb300 as G
    lib_kind = {"radau": G.ISDC_NODES_RADAU_RIGHT, "legendre": G.ISDC_NODES_GAUSS_LEGENDRE}[kind]
    orc_kind = {"radau": O.NODES_RADAU_RIGHT, "legendre": O.NODES_LEGENDRE}[kind]
    tau, Q, S = G.isdc_collocation_tables(M, nodes=lib_kind)
    np.testing.assert_allclose(tau, O.nodes(M, orc_kind), rtol=0, atol=2e-16)
    Qo = O.q_matrix(M, orc_kind)
    np.testing.assert_allclose(Q, Qo, rtol=0, atol=2e-15)
    np.testing.assert_allclose(S, np.diff(np.vstack([np.zeros(M), Qo]), axis=0), rtol=0, atol=2e-15)


def test_host_validation_without_gpu():
    import paper_1401_7824_gb300 as G
    with pytest.raises(G.IsdcError) as e:
        G.isdc_collocation_tables(3, nodes=3)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG
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
    assert (o.temporal_blocking, o.rb_run, o.stencil, o.equation, o.fused_transfer) == (-1, 0, 0, 0, -1)
    # option values outside their sets are refused before any device work
    for field, bad in [("rb_run", 3), ("rb_run", -16), ("rb_run", 64), ("temporal_blocking", 3),
                       ("smoother", 2), ("nu1", 17), ("stencil", 2), ("reaction", 5), ("max_sweeps", 0),
                       ("fused_transfer", 2), ("fused_transfer", -2), ("use_graphs", 3), ("use_graphs", -1)]:
        o = G.isdc_default_options()
        setattr(o, field, bad)
        with pytest.raises(G.IsdcError) as e:
            G.isdc_create(3, 31, 0.1, 3, 0.05, o)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG, field
        if field in ("use_graphs", "smoother"):  # the batch engine checks them before any device work too
            with pytest.raises(G.IsdcError) as e:
                G.isdc_batch_create(3, 31, 3, 1 << 30, 2, o)
            assert e.value.status == G.ISDC_ERR_INVALID_ARG, field
    o = G.isdc_default_options()
    o.equation = 1
    with pytest.raises(G.IsdcError) as e:
        G.isdc_create(2, 31, 0.1, 3, 0.05, o)  # periodic sides are 2^j
    assert e.value.status == G.ISDC_ERR_INVALID_ARG


def test_barrier_selftest_arguments_are_refused_before_device_work():
    """The grid-barrier self-test checks its arguments before any CUDA call."""
    import paper_1401_7824_gb300 as G
    lib = G.load()
    failed = ctypes.c_int(7)
    for blocks, phantom, limit in [(0, 0, 0.1), (2000, 0, 0.1), (4, -1, 0.1), (4, 2000, 0.1), (4, 0, 0.0),
                                   (4, 0, 11.0), (4, 0, float("nan"))]:
        st = lib.isdc_batch_barrier_selftest(blocks, phantom, limit, ctypes.byref(failed))
        assert st == G.ISDC_ERR_INVALID_ARG, (blocks, phantom, limit)
    assert lib.isdc_batch_barrier_selftest(4, 0, 0.1, None) == G.ISDC_ERR_INVALID_ARG
    assert failed.value == 7


def test_oversized_grids_and_bad_damping_are_refused_before_device_work():
    """Sides whose hierarchy would need more than 12 multigrid levels (2D 16383,
    32767) and Jacobi damping outside (0, 1] are refused by argument checks that
    run before any CUDA call, so they are exercised here without a GPU."""
    import paper_1401_7824_gb300 as G
    lib = G.load()
    dummy = ctypes.c_void_p(4096)  # never dereferenced: every call below fails its checks first
    for d, n in [(2, 16383), (2, 32767), (3, 255), (2, 2047), (3, 2047)]:
        st = lib.isdc_vcycles_static(d, n, 0.01, G.ISDC_SMOOTHER_JACOBI, 1, 1, 2.0 / 3.0, dummy, dummy, 1, None)
        assert st == G.ISDC_ERR_SCRATCH_TOO_SMALL, (d, n, st)
    for omega in [0.0, -0.5, 1.5, float("nan"), float("inf")]:
        st = lib.isdc_vcycles_static(2, 31, 0.01, G.ISDC_SMOOTHER_JACOBI, 1, 1, omega, dummy, dummy, 1, None)
        assert st == G.ISDC_ERR_INVALID_ARG, omega
        o = G.isdc_default_options()
        o.omega = omega
        with pytest.raises(G.IsdcError) as e:
            G.isdc_create(2, 31, 0.1, 3, 0.05, o)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG and "omega" in G.isdc_last_error()
        with pytest.raises(G.IsdcError) as e:
            G.isdc_batch_create(2, 31, 3, 1 << 30, 2, o)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG
    for n in [16383, 32767]:
        with pytest.raises(G.IsdcError) as e:
            G.isdc_create(2, n, 0.1, 3, 0.05)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG and "levels" in G.isdc_last_error()
        with pytest.raises(G.IsdcError) as e:
            G.isdc_batch_create(2, n, 3, 1 << 30, 2)
        assert e.value.status == G.ISDC_ERR_INVALID_ARG
    o = G.isdc_default_options()
    o.equation = 1
    with pytest.raises(G.IsdcError) as e:
        G.isdc_create(2, 16384, 0.1, 3, 0.05, o)
    assert e.value.status == G.ISDC_ERR_INVALID_ARG and "levels" in G.isdc_last_error()


@pytest.mark.parametrize("struct", ["isdc_options", "isdc_problem", "isdc_slot_info", "isdc_batch_info",
                                    "isdc_kernel_stat"])
def test_binding_structs_match_the_header_layout(struct, tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's size and
    field offsets (a layout mismatch would silently misread every option)."""
    import paper_1401_7824_gb300.isdc as B
    cls = getattr(B, struct)
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"isdc.h\"\nint main(void){\n"
                   + f'printf("%zu\\n", sizeof({struct}));\n'
                   + "".join(f'printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]
