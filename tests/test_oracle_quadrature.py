"""Pins for the oracle's collocation tables (Sec. 2, Eq. 2): Gauss-Lobatto
nodes, the integration matrix Q and the node-to-node matrix S."""
import numpy as np
import pytest

import oracle as O
from golden_io import lobatto_iiia_m3, lobatto_rules


@pytest.mark.parametrize("M", [3, 5, 7])
def test_lobatto_nodes_match_closed_form(M):
    nodes, weights = lobatto_rules()[M]
    np.testing.assert_allclose(O.lobatto_nodes(M), nodes, rtol=0, atol=1e-15)
    # the last row of Q is the full-interval quadrature rule
    np.testing.assert_allclose(O.q_matrix(M)[-1], weights, rtol=0, atol=2e-15)


def test_q_matrix_m3_is_lobatto_iiia_tableau():
    np.testing.assert_allclose(O.q_matrix(3), lobatto_iiia_m3(), rtol=0, atol=1e-15)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7])
def test_q_rows_integrate_polynomials_exactly(M):
    # Each row m integrates any polynomial of degree <= M-1 over [0, tau_m]
    # exactly, because Q interpolates on M nodes.
    tau = O.lobatto_nodes(M)
    Q = O.q_matrix(M)
    for p in range(M):
        np.testing.assert_allclose(Q @ tau ** p, tau ** (p + 1) / (p + 1), rtol=0, atol=1e-14)
    # The full row is the Lobatto rule: exact up to degree 2M-3.
    for p in range(2 * M - 2):
        assert abs(Q[-1] @ tau ** p - 1.0 / (p + 1)) < 1e-14
    # ... and not beyond (degree 2M-2 is not integrated exactly).
    assert abs(Q[-1] @ tau ** (2 * M - 2) - 1.0 / (2 * M - 1)) > 1e-9


@pytest.mark.parametrize("M", [3, 5, 7])
def test_s_matrix_is_node_to_node(M):
    tau = O.lobatto_nodes(M)
    S = O.s_matrix(M)
    assert S.shape == (M - 1, M)
    # row sums: integral of 1 from tau_m to tau_{m+1}
    np.testing.assert_allclose(S.sum(axis=1), np.diff(tau), rtol=0, atol=1e-15)
    # telescoping back to Q
    np.testing.assert_allclose(np.cumsum(S, axis=0), O.q_matrix(M)[1:], rtol=0, atol=1e-15)
    # S integrates tau^p over [tau_m, tau_{m+1}] exactly for p <= M-1
    for p in range(M):
        np.testing.assert_allclose(S @ tau ** p, np.diff(tau ** (p + 1)) / (p + 1), atol=1e-14)


# --- Gauss-Radau (right) and Gauss-Legendre nodes ------------------------------
FAMILIES = {"radau": O.NODES_RADAU_RIGHT, "legendre": O.NODES_LEGENDRE}


@pytest.mark.parametrize("fam,M", [("radau", 2), ("radau", 3), ("legendre", 2), ("legendre", 3)])
def test_radau_legendre_rules_match_closed_form(fam, M):
    from golden_io import collocation_tableaus, radau_legendre_rules
    nodes, weights = radau_legendre_rules()[(fam, M)]
    np.testing.assert_allclose(O.nodes(M, FAMILIES[fam]), nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.end_weights(M, FAMILIES[fam]), weights, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.q_matrix(M, FAMILIES[fam]), collocation_tableaus()[(fam, M)], rtol=0, atol=2e-15)


@pytest.mark.parametrize("fam", ["radau", "legendre"])
@pytest.mark.parametrize("M", [2, 3, 4, 5, 6, 7])
def test_radau_legendre_exactness(fam, M):
    """Q rows integrate degree <= M-1 exactly on [0, tau_m]; the full-step
    weights integrate up to degree 2M-2 (Radau) / 2M-1 (Gauss) and no further."""
    kind = FAMILIES[fam]
    tau, Q, w = O.nodes(M, kind), O.q_matrix(M, kind), O.end_weights(M, kind)
    assert np.all(np.diff(tau) > 0) and tau[0] > 0
    if fam == "radau":
        assert tau[-1] == 1.0
        np.testing.assert_allclose(Q[-1], w, rtol=0, atol=1e-15)
    else:
        assert tau[-1] < 1.0
        np.testing.assert_allclose(tau + tau[::-1], 1.0, rtol=0, atol=1e-15)  # symmetric
    for p in range(M):
        np.testing.assert_allclose(Q @ tau ** p, tau ** (p + 1) / (p + 1), rtol=0, atol=1e-14)
    top = 2 * M - 2 if fam == "radau" else 2 * M - 1
    for p in range(top + 1):
        assert abs(w @ tau ** p - 1.0 / (p + 1)) < 1e-14
    assert abs(w @ tau ** (top + 1) - 1.0 / (top + 2)) > 1e-9
