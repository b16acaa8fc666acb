"""Entry-by-entry pins of the oracle's reference matrices at every degree (no GPU).

Every matrix the oracle's discretisation is built from (Eq. bilinear_HDG_upwind
on the reference triangle) is recomputed here from an independent floating-point
Lagrange basis (monomial Vandermonde solve) and Gauss rules of sufficient
degree, and compared entry by entry: M, each barycentric-weighted mass ML[i],
the derivative matrices Dxi and Deta, the edge masses E[i], the cell-trace
couplings N[i] and the trace mass M1.  A mistake that keeps row and column sums
(a swapped pair of derivative entries, a wrong node order at p >= 3) fails here.
"""
import numpy as np
import pytest

from oracle import reference as ref
from tests.quadrature import FloatLagrange, float_trace_basis, gauss_segment, triangle_rule

VERTS = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])


def _close(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= 1e-12 * scale


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cell_matrices_entrywise(p):
    R = ref.reference_matrices(p)
    B = FloatLagrange(p)
    xi, eta, w = triangle_rule(p + 4)          # exact for the degree-(2p+1) integrands
    phi = B.values(xi, eta)
    assert _close(R["M"], (phi * w[:, None]).T @ phi)
    bary = [1.0 - xi - eta, xi, eta]
    for i in range(3):
        assert _close(R["ML"][i], (phi * (w * bary[i])[:, None]).T @ phi), f"ML[{i}]"
    # Dxi[a, b] = int phi_a d_xi phi_b, Deta likewise
    assert _close(R["Dxi"], (phi * w[:, None]).T @ B.d_xi(xi, eta))
    assert _close(R["Deta"], (phi * w[:, None]).T @ B.d_eta(xi, eta))
    # a transposed derivative matrix would not pass: the two orientations differ
    assert not _close(R["Dxi"].T, (phi * w[:, None]).T @ B.d_xi(xi, eta))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_edge_matrices_entrywise(p):
    R = ref.reference_matrices(p)
    B = FloatLagrange(p)
    t, w = gauss_segment(p + 2)
    mu = float_trace_basis(p, t)
    assert _close(R["M1"], (mu * w[:, None]).T @ mu)
    for i in range(3):
        # local edge i runs from vertex (i+1)%3 to (i+2)%3, parameter t in [0, 1]
        A, Bv = VERTS[(i + 1) % 3], VERTS[(i + 2) % 3]
        pts = A[None, :] + t[:, None] * (Bv - A)[None, :]
        phi = B.values(pts[:, 0], pts[:, 1])
        assert _close(R["E"][i], (phi * w[:, None]).T @ phi), f"E[{i}]"
        assert _close(R["N"][i], (phi * w[:, None]).T @ mu), f"N[{i}]"


@pytest.mark.parametrize("p", [3, 4])
def test_cell_basis_values_at_interior_points(p):
    """The oracle's basis evaluation agrees with the independent one away from the nodes."""
    rng = np.random.default_rng(p)
    u = rng.random((50, 2))
    xi, eta = np.where(u.sum(1) > 1, 1 - u[:, 0], u[:, 0]), np.where(u.sum(1) > 1, 1 - u[:, 1], u[:, 1])
    assert np.abs(ref.eval_cell_basis(p, xi, eta) - FloatLagrange(p).values(xi, eta)).max() < 1e-12


def test_a_sum_preserving_mistake_is_caught():
    """Plant, in a copy of the oracle's p = 3 derivative matrix, a change that
    keeps every row and column sum (what the divergence-theorem checks see):
    the entry-by-entry comparison rejects it."""
    p = 3
    R = ref.reference_matrices(p)
    D = R["Dxi"].copy()
    eps = 1e-3
    D[0, 0] += eps; D[1, 1] += eps; D[0, 1] -= eps; D[1, 0] -= eps
    assert np.allclose(D.sum(axis=0), R["Dxi"].sum(axis=0)) and np.allclose(D.sum(axis=1), R["Dxi"].sum(axis=1))
    B = FloatLagrange(p)
    xi, eta, w = triangle_rule(p + 4)
    assert not _close(D, (B.values(xi, eta) * w[:, None]).T @ B.d_xi(xi, eta))
