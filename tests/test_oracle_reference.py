"""Pins of the oracle's reference-element algebra (no GPU).

The exact monomial integration of the oracle is compared with an independent
collapsed Gauss rule, and with closed forms: the triangle area, the annihilation
of constants by derivatives, partitions of unity, and the known P1 element
matrices.
"""
import numpy as np
import pytest

from oracle import reference as ref
from tests.quadrature import triangle_rule


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_matrix_against_gauss_rule(p):
    R = ref.reference_matrices(p)
    xi, eta, w = triangle_rule(p + 3)
    phi = ref.eval_cell_basis(p, xi, eta)
    M_q = (phi * w[:, None]).T @ phi
    assert np.allclose(R["M"], M_q, atol=1e-14, rtol=0)
    assert abs(R["M"].sum() - 0.5) < 1e-14                       # area of the reference cell


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_property_and_derivatives(p):
    nodes = ref.cell_nodes(p)
    phi = ref.eval_cell_basis(p, nodes[:, 0], nodes[:, 1])
    assert np.allclose(phi, np.eye(len(nodes)), atol=1e-12)
    R = ref.reference_matrices(p)
    # derivative of the constant sum_b phi_b = 1 vanishes
    assert np.allclose(R["Dxi"].sum(axis=1), 0, atol=1e-13)
    assert np.allclose(R["Deta"].sum(axis=1), 0, atol=1e-13)
    # int d_xi phi_b over the triangle = boundary integral of phi_b * n_xi (divergence theorem)
    lengths = [np.sqrt(2.0), 1.0, 1.0]
    nxi = [1 / np.sqrt(2.0), -1.0, 0.0]
    bnd = sum(lengths[i] * nxi[i] * R["E"][i].sum(axis=0) for i in range(3))
    assert np.allclose(R["Dxi"].sum(axis=0), bnd, atol=1e-13)
    # barycentric-weighted masses add up to the mass matrix
    assert np.allclose(sum(R["ML"]), R["M"], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_trace_matrices(p):
    R = ref.reference_matrices(p)
    # 1-D mass of the equispaced Lagrange basis on [0,1] sums to the length
    assert abs(R["M1"].sum() - 1.0) < 1e-14
    for i in range(3):
        # partition of unity: sum_j mu_j = 1, sum_b phi_b = 1 on the edge
        assert np.allclose(R["N"][i].sum(axis=1), R["E"][i].sum(axis=1), atol=1e-14)
        assert abs(R["E"][i].sum() - 1.0) < 1e-14
        # the cell basis restricted to its edge is in P^p(e): N maps it exactly
        # onto the trace basis, so E = N M1^-1 N^T
        assert np.allclose(R["E"][i], R["N"][i] @ np.linalg.solve(R["M1"], R["N"][i].T), atol=1e-13)


def test_p1_closed_form():
    R = ref.reference_matrices(1)
    assert np.allclose(R["M"], (np.ones((3, 3)) + np.eye(3)) / 24.0, atol=1e-15)
