"""Pins of the oracle's iterative solver (no GPU).

* GMRES: finite termination on a small nonsymmetric system and agreement with
  the direct solution (the exact result it must reach);
* P1 spaces (Sec. 4.4, upwind coarse space): closed forms of the assembled
  mass and stiffness matrices;
* the geometric P1 V-cycle is a convergent iteration;
* Alg. twolevel_vcycle as a preconditioner: for f = 0 the preconditioned
  operator has its spectrum bounded away from zero uniformly in h (the
  h-robustness the paper reports for this method), and the two-level
  error propagation is a contraction in the energy norm;
* the damped block-Jacobi smoother is convergent;
* the cell matrices (momentum rows scaled by H/g) have a positive-definite
  symmetric part up to Courant 16, so an LU without pivoting exists.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle.hdg import HDGProblem, MeshData
from oracle.solver import (gmres, p1_matrices, TwoLevelPreconditioner, P1Multigrid,
                           nested_prolongation, solve_iterative)


def test_gmres_finite_termination():
    rng = np.random.default_rng(0)
    n = 12
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n)
    x, info = gmres(lambda v: A @ v, b, restart=n, rtol=1e-13)
    assert info["iters"] <= n
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-11


def test_gmres_restarted_with_preconditioner():
    rng = np.random.default_rng(1)
    n = 60
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 3 * np.eye(n)
    b = rng.standard_normal(n)
    Minv = np.linalg.inv(np.diag(np.diag(A)))
    x, info = gmres(lambda v: A @ v, b, precond=lambda v: Minv @ v, restart=5, rtol=1e-12)
    assert info["converged"]
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_p1_matrices_closed_forms(kind):
    mesh = I.periodic_square(6, side=2.0) if kind == "flat" else I.icosahedral_sphere(2)
    Mm, Km = p1_matrices(MeshData.of(mesh))
    ones = np.ones(mesh.n_vertices)
    area = ones @ Mm @ ones
    if kind == "flat":
        assert abs(area - 4.0) < 1e-13
    else:
        assert 0.9 * 4 * np.pi < area < 4 * np.pi          # flat facets inside the sphere
    assert np.abs(Km @ ones).max() < 1e-12
    assert np.abs((Km - Km.T).toarray()).max() < 1e-14
    # stiffness of x on the flat mesh: a(x, x) = |grad x|^2 * area on one period is not
    # periodic, so use sin: a(sin, sin) ~ k^2 * int sin^2 for a fine mesh
    if kind == "flat":
        mesh2 = I.periodic_square(64)
        M2, K2 = p1_matrices(MeshData.of(mesh2))
        k = 2 * np.pi
        v = np.sin(k * mesh2.vertex_xyz[:, 0])
        assert (v @ K2 @ v) / (v @ M2 @ v) == pytest.approx(k * k, rel=2e-3)


def _flat(n, p=1, tau=None, f0=0.0, g=1.0, H=1.0, courant=8.0):
    mesh = I.periodic_square_hierarchy(n, n_coarsest=4)
    tau = courant * mesh.h if tau is None else tau
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=I.coriolis_flat(mesh, f0))
    return mesh, prob


def test_p1_vcycle_converges():
    mesh, prob = _flat(16)
    pc = TwoLevelPreconditioner(prob, mesh, prob.trace_operator())
    mg = pc.mg
    A = mg.ops[0].toarray()
    n = A.shape[0]
    E = np.eye(n) - np.stack([mg.vcycle(A[:, j]) for j in range(n)], axis=1)
    assert np.abs(np.linalg.eigvals(E)).max() < 0.5


def _dense_pc(pc, n):
    return np.stack([pc(np.eye(n)[:, j]) for j in range(n)], axis=1)


@pytest.mark.parametrize("coarse", ["exact", "gmg"])
def test_two_level_spectrum_h_robust(coarse):
    mins = []
    for n in (4, 8, 16):
        mesh, prob = _flat(n)
        S = prob.trace_operator()
        pc = TwoLevelPreconditioner(prob, mesh, S, coarse=coarse)
        Sd = S.toarray()
        V = _dense_pc(pc, Sd.shape[0])
        ev = np.linalg.eigvals(V @ Sd)
        mins.append(np.abs(ev).min())
        # energy-norm contraction of I - V S  (S SPD for f = 0)
        L = np.linalg.cholesky(Sd)
        Eg = np.eye(Sd.shape[0]) - V @ Sd
        assert np.linalg.norm(L.T @ Eg @ np.linalg.inv(L.T), 2) < 1.0
    assert min(mins) > 0.3
    assert max(mins) / min(mins) < 1.5


def test_block_jacobi_is_convergent():
    mesh, prob = _flat(8, p=2)
    S = prob.trace_operator()
    pc = TwoLevelPreconditioner(prob, mesh, S)
    G = np.eye(S.shape[0]) - pc.omega * (pc.Dinv @ S).toarray()
    assert np.abs(np.linalg.eigvals(G)).max() < 1.0


@pytest.mark.parametrize("p,courant", [(1, 16.0), (3, 16.0), (4, 4.0)])
def test_scaled_cell_matrix_has_pd_symmetric_part(p, courant):
    g, H = 9.81, 1.0e3
    c = np.sqrt(g * H)
    mesh = I.periodic_square(4, side=4 * 2.0e4)
    tau = courant * mesh.h / c
    prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=I.coriolis_flat(mesh, 1e-4))
    n = prob.np
    D = np.diag(np.r_[np.full(2 * n, H / g), np.ones(n)])
    for K in range(prob.N):
        A = D @ prob.ops[K][0]
        assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_iterative_solve_reaches_direct_solution(kind):
    if kind == "flat":
        mesh, prob = _flat(8, p=2, f0=1.0)
    else:
        mesh = I.sphere_hierarchy(2, 1.0, r_coarsest=0)
        prob = HDGProblem(mesh, 2, tau=8 * mesh.h, g=1.0, H=1.0, f_vertex=I.coriolis_sphere(mesh, 0.5))
    rng = np.random.default_rng(7)
    ru = rng.standard_normal((prob.N, 2, prob.np))
    rh = rng.standard_normal((prob.N, prob.np))
    (u, h), lam, info = solve_iterative(prob, mesh, ru, rh, rtol=1e-12)
    (u0, h0), lam0 = prob.solve_condensed(ru, rh)
    assert info["converged"] and info["iters"] < 40
    assert np.linalg.norm(lam - lam0) / np.linalg.norm(lam0) < 1e-10
    assert np.linalg.norm(h - h0) / np.linalg.norm(h0) < 1e-10


# ---------------------------------------------------------------------------
# coarse operator with the implicit Coriolis term (reading of Sec. 4.4)

def test_rotating_coarse_operator_reduces_to_the_printed_form_without_rotation():
    from oracle.solver import p1_rotating_operator
    mesh = I.icosahedral_sphere(2)
    md = MeshData.of(mesh)
    tau, g, H = 0.3, 1.7, 0.6
    A = p1_rotating_operator(md, np.zeros(mesh.n_vertices), tau, g, H)
    Mm, Km = p1_matrices(md)
    B = (Mm + tau * tau * g * H * Km) / tau
    assert np.abs((A - B).toarray()).max() <= 1e-13 * np.abs(B.toarray()).max()


def test_rotating_coarse_operator_constant_f_has_no_skew_part():
    """On a closed surface with constant f the skew term sums to zero for P1
    (tangential derivatives are continuous), leaving kappa = 1/(1+tau^2 f^2)."""
    from oracle.solver import p1_rotating_operator
    mesh = I.periodic_square(8)
    md = MeshData.of(mesh)
    tau, g, H, f0 = 0.4, 1.0, 2.0, 3.0
    A = p1_rotating_operator(md, np.full(mesh.n_vertices, f0), tau, g, H).toarray()
    Mm, Km = p1_matrices(md)
    kap = 1.0 / (1.0 + (tau * f0) ** 2)
    B = ((Mm + tau * tau * g * H * kap * Km) / tau).toarray()
    assert np.abs(A - B).max() <= 1e-12 * np.abs(B).max()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()


def test_rotating_coarse_operator_fourier_symbol():
    """A smooth Fourier mode sees the continuum symbol (1 + tau^2 g H k^2 / (1 + tau^2 f^2)) / tau."""
    from oracle.solver import p1_rotating_operator
    n = 64
    mesh = I.periodic_square(n)
    md = MeshData.of(mesh)
    tau, g, H, f0 = 0.05, 1.0, 1.0, 25.0
    A = p1_rotating_operator(md, np.full(mesh.n_vertices, f0), tau, g, H)
    Mm, _ = p1_matrices(md)
    k = 2 * np.pi
    x = np.cos(k * mesh.vertex_xyz[:, 0])
    ratio = (x @ A @ x) / (x @ Mm @ x)
    expect = (1 + tau * tau * g * H * k * k / (1 + (tau * f0) ** 2)) / tau
    assert ratio == pytest.approx(expect, rel=2e-3)


def test_rotating_coarse_operator_helps_under_rotation():
    """Sphere, f tau ~ 2: the coarse problem with rotation needs fewer FGMRES
    iterations than the rotation-free one; both converge (a check of the
    reading, not a value printed in the paper)."""
    R, om = 6.371e6, 7.292e-5
    mesh = I.sphere_hierarchy(4, R, r_coarsest=1)
    g, H = 9.81, 7500.0
    tau = 8.0 * mesh.h / np.sqrt(g * H)
    f = I.coriolis_sphere(mesh, om)
    prob = HDGProblem(mesh, 1, tau=tau, g=g, H=H, f_vertex=f)
    rng = np.random.default_rng(3)
    ru = rng.standard_normal((prob.N, 2, prob.np))
    rh = rng.standard_normal((prob.N, prob.np))
    its = {}
    for mode in ("rotating", "rediscretised"):
        _, _, info = solve_iterative(prob, mesh, ru, rh, rtol=1e-8, coarse_mode=mode)
        assert info["converged"]
        its[mode] = info["iters"]
    assert its["rotating"] < its["rediscretised"]
