"""Pins of the Lax-Friedrichs oracle (oracle/lf.py; Eq. bilinear_HDG_lax, the
RT0 coarse space and Eq. coarse_problem_LF of Sec. 4.4), no GPU.

1. monolithic solve == condensed solve (the Schur reduction is exact);
2. energy identity u_hat^T S u_hat = (1/tau)(||u||^2 + (g/H)||h||^2)
   + tau_s sum_K ||u - u_hat||^2_dK for the local responses; S symmetric
   positive definite for f = 0, positive real with asymmetry linear in f;
3. exact mass conservation;
4. manufactured convergence at order >= p + 1/2, p = 1..3;
5. the Lax-Friedrichs and upwind solutions converge to each other;
6. RT0 transfer: pi reproduces constant vector fields and RT0 fields exactly
   at every trace node; the divergence of each RT0 basis function integrates
   to its boundary flux; the coarse operator's scale: on smooth fields
   (pi u_c)^T S (pi u_c) / u_c^T S_c u_c -> 1;
7. the two-level preconditioner's iteration count levels off as 1/h grows.
"""
import numpy as np
import pytest

import hdg_inputs as I
from oracle import reference as ref
from oracle.hdg import HDGProblem, cell_geometry
from oracle.lf import (LFProblem, LFTwoLevelPreconditioner, facet_normals, rt0_cell_basis, rt0_injection,
                       rt0_operator)
from oracle.solver import gmres
from tests.test_oracle_pins import _l2_error


def _prob(p=2, f0=0.0, n=4, tau=0.3, g=1.3, H=0.7):
    mesh = I.periodic_square(n)
    return mesh, LFProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=I.coriolis_flat(mesh, f0))


def _rhs(prob, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((prob.N, 2, prob.np)), rng.standard_normal((prob.N, prob.np))


@pytest.mark.parametrize("p,f0", [(1, 0.0), (2, 1.0), (3, 0.5)])
def test_monolithic_equals_condensed(p, f0):
    mesh, prob = _prob(p, f0)
    ru, rh = _rhs(prob, 1)
    (u1, h1), l1 = prob.solve_monolithic(ru, rh)
    (u2, h2), l2 = prob.solve_condensed(ru, rh)
    sc = max(np.abs(u1).max(), np.abs(h1).max())
    assert np.abs(u1 - u2).max() <= 1e-12 * sc and np.abs(h1 - h2).max() <= 1e-12 * sc
    assert np.abs(l1 - l2).max() <= 1e-12 * np.abs(l1).max()


def _edge_mismatch2(prob, K, uK, lK):
    """sum over the edges of K of int_e |u - u_hat|^2."""
    R = ref.reference_matrices(prob.prm.p)
    _, _, lengths, _ = cell_geometry(prob.X[K])
    pp = prob.prm.p + 1
    s = 0.0
    for i in range(3):
        for c in range(2):
            l = lK[i * 2 * pp + c * pp:i * 2 * pp + (c + 1) * pp]
            s += lengths[i] * (uK[c] @ R["E"][i] @ uK[c] - 2 * uK[c] @ R["N"][i] @ l + l @ R["M1"] @ l)
    return s


@pytest.mark.parametrize("p,f0", [(1, 0.0), (2, 0.0), (3, 0.0), (2, 1.5)])
def test_energy_identity(p, f0):
    mesh, prob = _prob(p, f0)
    S = prob.trace_operator().toarray()
    n = prob.np
    prm = prob.prm
    for lam in np.random.default_rng(3).standard_normal((3, prob.n_trace)):
        lhs = lam @ S @ lam
        eu = eh = eb = 0.0
        for K in range(prob.N):
            A, B, C, Mt, Mass = prob.op(K)
            lK = lam[prob.gdof[K]]
            q = -np.linalg.solve(A, B @ lK)
            Mk = Mass[:n, :n]
            eu += q[:n] @ Mk @ q[:n] + q[n:2 * n] @ Mk @ q[n:2 * n]
            eh += q[2 * n:] @ Mk @ q[2 * n:]
            eb += _edge_mismatch2(prob, K, (q[:n], q[n:2 * n]), lK)
        rhs = (eu + (prm.g / prm.H) * eh) / prm.tau + prm.tau_s * eb
        assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    asym = np.abs(S - S.T).max() / np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    if f0 == 0.0:
        assert asym <= 1e-13
    else:
        assert asym > 1e-6


def test_asymmetry_scales_with_rotation():
    vals = []
    for f0 in (0.01, 0.02, 0.04):
        _, prob = _prob(1, f0)
        S = prob.trace_operator().toarray()
        vals.append(np.abs(S - S.T).max())
    assert vals[1] / vals[0] == pytest.approx(2.0, rel=0.01) and vals[2] / vals[1] == pytest.approx(2.0, rel=0.01)


@pytest.mark.parametrize("p", [1, 3])
def test_mass_conservation(p):
    mesh, prob = _prob(p, 1.0)
    ru, rh = _rhs(prob, 4)
    (u, h), _ = prob.solve_condensed(ru, rh)
    assert abs(prob.integral_of_h(h) - prob.integral_of_h(rh)) <= 1e-12 * prob.integral_of_h(np.abs(rh))


def _manufactured(p, n, flux):
    mesh = I.periodic_square(n)
    tau = 8 * mesh.h
    cls = LFProblem if flux == "lf" else HDGProblem
    prob = cls(mesh, p, tau=tau, g=1.0, H=1.0, f_vertex=I.coriolis_flat(mesh, 1.0), tau_s=1.0)
    ru, rh = I.manufactured_rhs(mesh, p, tau, 1.0, 1.0, 1.0)
    (u, h), _ = prob.solve_condensed(ru, rh)
    return mesh, prob, u, h


@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_convergence(p):
    errs = []
    for n in (4, 8, 16):
        mesh, prob, u, h = _manufactured(p, n, "lf")
        errs.append(_l2_error(prob, mesh, u, h, lambda x: I.fields.manufactured_solution(x, 1.0, 1.0, 1.0)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates[-1] >= p + 0.5).all(), rates


def test_lax_friedrichs_and_upwind_agree_in_the_limit():
    diffs = []
    for n in (4, 8, 16):
        _, prob, u1, h1 = _manufactured(2, n, "lf")
        _, _, u2, h2 = _manufactured(2, n, "up")
        diffs.append(np.sqrt(prob.l2_norm2_cells(h1 - h2)))
    assert diffs[2] < diffs[1] < diffs[0] and diffs[1] / diffs[2] > 4


def _rt0_interpolant(prob, field):
    """Normal component of a vector field at the facet midpoints (RT0 dofs)."""
    nu = facet_normals(prob)
    mids = np.zeros((prob.n_facets, 2))
    for K in range(prob.N):
        for i in range(3):
            mids[prob.facet_of[K, i]] = 0.5 * (prob.X[K, (i + 1) % 3] + prob.X[K, (i + 2) % 3])
    return np.einsum("ec,ec->e", field(mids), nu)


def test_rt0_injection_reproduces_constant_fields():
    mesh, prob = _prob(2, 0.0)
    Pi = rt0_injection(prob).toarray()
    for vec in ((1.0, 0.0), (0.3, -2.0)):
        c = _rt0_interpolant(prob, lambda x: np.broadcast_to(np.array(vec), x.shape))
        x = Pi @ c
        pp = prob.prm.p + 1
        for comp in range(2):
            vals = x.reshape(prob.n_facets, 2, pp)[:, comp, :]
            assert np.abs(vals - vec[comp]).max() <= 1e-13


def test_rt0_basis_divergence_and_normal_components():
    mesh, prob = _prob(1, 0.0)
    for K in range(5):
        X = prob.X[K]
        detJ, _, lengths, normals = cell_geometry(X)
        for i in range(3):
            for j in range(3):
                # normal component of phi_i on edge j: 1 on edge i, 0 elsewhere (two points per edge)
                a, b = X[(j + 1) % 3], X[(j + 2) % 3]
                pts = np.stack([a + 0.2 * (b - a), a + 0.7 * (b - a)])
                assert np.allclose(rt0_cell_basis(X, i, pts) @ normals[j], 1.0 if i == j else 0.0, atol=1e-13)
            # div phi_i = |e_i| / |K|: its integral equals the boundary flux |e_i|
            assert 2 * lengths[i] / detJ * (0.5 * detJ) == pytest.approx(lengths[i])


def test_coarse_scale_on_smooth_fields():
    """(pi u_c)^T S (pi u_c) / u_c^T S_c u_c tends to 1 on smooth fields."""
    ratios = []
    for n in (8, 16):
        mesh = I.periodic_square(n)
        prob = LFProblem(mesh, 2, tau=8 * mesh.h, g=1.0, H=1.0, f_vertex=np.zeros(mesh.n_vertices))
        S, Pi, Sc = prob.trace_operator(), rt0_injection(prob), rt0_operator(prob)
        k = 2 * np.pi * np.array([1.0, 0.0])
        c = _rt0_interpolant(prob, lambda x: np.stack([np.cos(x @ k), 0.5 * np.sin(x @ k)], axis=-1))
        x = Pi @ c
        ratios.append((x @ (S @ x)) / (c @ (Sc @ c)))
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1) and abs(ratios[1] - 1) < 0.1


def test_two_level_iterations_are_h_robust():
    its = []
    for n in (8, 16, 32):
        mesh = I.periodic_square(n)
        prob = LFProblem(mesh, 1, tau=2 * mesh.h, g=1.0, H=1.0, f_vertex=I.coriolis_flat(mesh, 0.5))
        S = prob.trace_operator()
        b = np.random.default_rng(0).standard_normal(S.shape[0])
        _, info = gmres(lambda v: S @ v, b, LFTwoLevelPreconditioner(prob, S), rtol=1e-8, maxiter=300)
        assert info["converged"]
        its.append(info["iters"])
    _, info0 = gmres(lambda v: S @ v, b, None, rtol=1e-8, maxiter=300)
    # the count levels off as the mesh is refined (38, 44, 45 here)
    assert its[2] - its[1] <= 2 and max(its) <= 1.25 * min(its)
    assert not info0["converged"] or info0["iters"] > 2 * max(its)
