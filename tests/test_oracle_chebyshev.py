"""Pins of the oracle's Chebyshev smoother (no GPU).

The smoother is the Chebyshev iteration for D^-1 S (D the facet diagonal
blocks) on an ellipse fitted to Arnoldi Ritz values (the paper smooths with
Chebyshev iterations, Sec. 5.2.1 and the solver configuration appendix).

* With delta^2 = 0 it is damped block-Jacobi with omega = 1/theta.
* Its error propagation after n steps is the scaled Chebyshev polynomial
  T_n((theta - mu)/delta) / T_n(theta/delta) of D^-1 S: checked on the
  eigenvectors of D^-1 S, for a real interval (f = 0) and for a tall ellipse
  (delta^2 < 0, strong rotation).
* Arnoldi run to the full dimension reproduces the eigenvalues; the fitted
  ellipse holds every Ritz value in its real range; a hand-computed fit.
* Under strong rotation (max |f| tau = 4.1), where damped block-Jacobi with
  omega = 2/3 makes the two-level method diverge, the Chebyshev smoother
  converges.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem
from oracle.solver import (TwoLevelPreconditioner, arnoldi_ritz, chebyshev_ellipse, chebyshev_polynomial,
                           chebyshev_start_vector, gmres)


def _small(f0=0.0, p=1):
    mesh = I.periodic_square_hierarchy(4, n_coarsest=2)
    prob = HDGProblem(mesh, p, tau=0.4, g=1.0, H=1.0, f_vertex=I.coriolis_flat(mesh, f0))
    return mesh, prob, prob.trace_operator().tocsr()


def test_zero_focal_distance_is_damped_jacobi():
    mesh, prob, S = _small(f0=1.0)
    b = np.random.default_rng(0).standard_normal(S.shape[0])
    pj = TwoLevelPreconditioner(prob, mesh, S, omega=1.0 / 1.3)
    pc = TwoLevelPreconditioner(prob, mesh, S, smoother="chebyshev", cheb=(1.3, 0.0))
    for n in (1, 2, 3):
        a, c = pj.smooth(b, np.zeros_like(b), n), pc.smooth(b, np.zeros_like(b), n)
        assert np.abs(a - c).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("f0,cheb", [(0.0, (1.1, 0.8)), (6.0, (1.2, -2.5))])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_error_propagation_is_the_chebyshev_polynomial(f0, cheb, n):
    mesh, prob, S = _small(f0=f0)
    pc = TwoLevelPreconditioner(prob, mesh, S, smoother="chebyshev", cheb=cheb)
    DS = (pc.Dinv @ S).toarray()
    mu, V = np.linalg.eig(DS)
    # error propagation of n steps with b = 0, column by column
    E = np.stack([pc.smooth(np.zeros(S.shape[0]), e, n) for e in np.eye(S.shape[0])], axis=1)
    pn = chebyshev_polynomial(mu, cheb[0], cheb[1], n)
    assert np.abs(E @ V - V * pn[None, :]).max() <= 1e-9 * max(1.0, np.abs(pn).max())


def test_full_arnoldi_gives_the_eigenvalues():
    mesh, prob, S = _small(f0=2.0)
    pc = TwoLevelPreconditioner(prob, mesh, S)
    DS = (pc.Dinv @ S).toarray()
    n = S.shape[0]
    ritz = arnoldi_ritz(lambda v: DS @ v, chebyshev_start_vector(n), n)
    ev = np.linalg.eigvals(DS)
    # every eigenvalue has a Ritz value next to it
    d = np.abs(ev[:, None] - ritz[None, :]).min(axis=1)
    assert d.max() <= 1e-8 * np.abs(ev).max()


def test_ellipse_fit():
    theta, delta2 = chebyshev_ellipse(np.array([1.0, 2.0, 0.5]))
    # b = 2.2, a = 0.22: centre 1.21, half-width 0.99, no imaginary extent
    assert theta == pytest.approx(1.21) and delta2 == pytest.approx(0.99 ** 2)
    ritz = np.array([0.3 + 0j, 1.0 + 1.5j, 1.0 - 1.5j, 1.8 + 0.4j, 1.8 - 0.4j, 2.0 + 0j, 0.05 + 0.01j])
    theta, delta2 = chebyshev_ellipse(ritz)
    b = 2.2
    a, A = 0.22, 0.99
    B2 = A * A - delta2
    assert theta == pytest.approx(0.5 * (a + b))
    inside = [((z.real - theta) / A) ** 2 + z.imag ** 2 / B2 for z in ritz if z.real >= a]
    assert max(inside) <= 1.0


def test_chebyshev_converges_under_strong_rotation():
    R, om = 6.371e6, 7.292e-5
    mesh = I.sphere_hierarchy(3, R, r_coarsest=1)
    g, H = 9.81, 7500.0
    tau = 8.0 * mesh.h / np.sqrt(g * H)
    f = I.coriolis_sphere(mesh, om)
    assert 4.0 < np.abs(f).max() * tau < 4.3
    prob = HDGProblem(mesh, 2, tau=tau, g=g, H=H, f_vertex=f)
    S = prob.trace_operator().tocsr()
    b = np.random.default_rng(0).standard_normal(S.shape[0])
    _, info_j = gmres(lambda v: S @ v, b, TwoLevelPreconditioner(prob, mesh, S), rtol=1e-8, maxiter=80)
    pc = TwoLevelPreconditioner(prob, mesh, S, smoother="chebyshev")
    assert pc.cheb[1] < 0                    # a tall ellipse: the rotation-dominated modes
    _, info_c = gmres(lambda v: S @ v, b, pc, rtol=1e-8, maxiter=80)
    assert not info_j["converged"]
    assert info_c["converged"] and info_c["iters"] <= 30
