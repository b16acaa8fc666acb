"""Pins of the oracle's HDG discretisation against facts fixed by the paper and
by the mathematics (no GPU).

1. monolithic solve == condensed solve (Sec. 4.2: the Schur-complement
   reduction is exact);
2. HDG (u, h) == standard upwind DG (u, h) (the equivalence stated after
   Eq. linear_hybridized), through a separately written assembly;
3. energy identity of the trace operator (from Eq. bilinear_HDG_upwind; the
   Cockburn-relation argument of Sec. 4.3 that S is positive definite);
4. exact discrete mass conservation;
5. manufactured-solution convergence at order >= p + 1/2 (Sec. 7.3);
6. Fourier-mode closed form on the periodic square (zero geometric error);
7. tau -> 0 limit and the P1 injection of Sec. 4.4;
8. dof counts of Tab. grid_setup and Tab. grid_setup_spherical.
"""
import json
import math
import os

import numpy as np
import pytest

import hdg_inputs as I
from oracle import reference as ref
from oracle.hdg import HDGProblem, cell_geometry
from oracle.stddg import solve_standard_dg
from oracle.solver import injection
from tests.quadrature import triangle_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_rhs(prob, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((prob.N, 2, prob.np)), rng.standard_normal((prob.N, prob.np))


def _problem(kind, p, tau=0.3, g=1.3, H=0.7, f0=1.0):
    if kind == "flat":
        mesh = I.periodic_square(4)
        f = I.coriolis_flat(mesh, f0)
    else:
        mesh = I.icosahedral_sphere(1, 1.0)
        f = I.coriolis_sphere(mesh, 0.5 * f0)
    return mesh, HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=f)


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 2), ("flat", 3), ("sphere", 1), ("sphere", 2)])
def test_monolithic_equals_condensed(kind, p):
    mesh, prob = _problem(kind, p)
    ru, rh = _rand_rhs(prob, 1)
    (u1, h1), l1 = prob.solve_monolithic(ru, rh)
    (u2, h2), l2 = prob.solve_condensed(ru, rh)
    scale = max(np.abs(u1).max(), np.abs(h1).max())
    assert np.abs(u1 - u2).max() <= 1e-12 * scale
    assert np.abs(h1 - h2).max() <= 1e-12 * scale
    assert np.abs(l1 - l2).max() <= 1e-12 * np.abs(l1).max()


@pytest.mark.parametrize("kind,p", [("flat", 1), ("flat", 2), ("flat", 3), ("flat", 4), ("sphere", 2)])
def test_hdg_equals_standard_dg(kind, p):
    mesh, prob = _problem(kind, p)
    ru, rh = _rand_rhs(prob, 2)
    (u1, h1), _ = prob.solve_condensed(ru, rh)
    u2, h2 = solve_standard_dg(prob, ru, rh)
    scale = max(np.abs(u1).max(), np.abs(h1).max())
    assert np.abs(u1 - u2).max() <= 1e-12 * scale
    assert np.abs(h1 - h2).max() <= 1e-12 * scale


def _edge_mismatch2(prob, K, hK, lamK):
    """sum over the edges of K of int_e (h - lambda)^2."""
    R = ref.reference_matrices(prob.prm.p)
    _, _, lengths, _ = cell_geometry(prob.X[K])
    pp = prob.prm.p + 1
    s = 0.0
    for i in range(3):
        l = lamK[i * pp:(i + 1) * pp]
        s += lengths[i] * (hK @ R["E"][i] @ hK - 2 * hK @ R["N"][i] @ l + l @ R["M1"] @ l)
    return s


@pytest.mark.parametrize("kind,p,f0", [("flat", 1, 0.0), ("flat", 2, 0.0), ("sphere", 2, 0.0),
                                        ("flat", 2, 1.0), ("sphere", 1, 3.0), ("flat", 3, 0.0),
                                        ("flat", 3, 1.0), ("sphere", 3, 0.0), ("flat", 4, 0.0)])
def test_energy_identity(kind, p, f0):
    """lambda^T S lambda = (1/tau)((H/g)||u||^2 + ||h||^2) + tau_s sum_K ||h - lambda||^2_dK
    for the local responses (u, h) to lambda with zero RHS; holds for any f
    because (u_perp, u) = 0 pointwise."""
    mesh, prob = _problem(kind, p, f0=f0)
    S = prob.trace_operator().toarray()
    rng = np.random.default_rng(3)
    prm = prob.prm
    n = prob.np
    for _ in range(3):
        lam = rng.standard_normal(prob.n_trace)
        lhs = lam @ S @ lam
        e_u = e_h = e_b = 0.0
        for K in range(prob.N):
            A, B, C, Mt, Mass = prob.ops[K]
            lK = lam[prob.gdof[K]]
            q = -np.linalg.solve(A, B @ lK)
            Mk = Mass[:n, :n]
            e_u += q[:n] @ Mk @ q[:n] + q[n:2 * n] @ Mk @ q[n:2 * n]
            e_h += q[2 * n:] @ Mk @ q[2 * n:]
            e_b += _edge_mismatch2(prob, K, q[2 * n:], lK)
        rhs = ((prm.H / prm.g) * e_u + e_h) / prm.tau + prm.tau_s * e_b
        assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    asym = np.abs(S - S.T).max() / np.abs(S).max()
    if f0 == 0.0:
        assert asym <= 1e-13
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    else:
        assert asym > 1e-6                     # rotation makes S nonsymmetric
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0   # but positive real


def test_asymmetry_scales_with_rotation():
    """To first order in f, ||S - S^T|| grows linearly with the rotation rate."""
    vals = []
    for f0 in (0.01, 0.02, 0.04):
        _, prob = _problem("flat", 1, f0=f0)
        S = prob.trace_operator().toarray()
        vals.append(np.abs(S - S.T).max())
    assert vals[1] / vals[0] == pytest.approx(2.0, rel=0.01)
    assert vals[2] / vals[1] == pytest.approx(2.0, rel=0.01)


@pytest.mark.parametrize("kind,p", [("flat", 2), ("sphere", 2), ("flat", 3), ("sphere", 3), ("flat", 4)])
def test_mass_conservation(kind, p):
    """psi = 1 on every cell plus mu = 1 on every facet: the facet fluxes cancel,
    so int h = int r_h exactly (up to roundoff) for the direct solve."""
    mesh, prob = _problem(kind, p)
    ru, rh = _rand_rhs(prob, 4)
    (u, h), _ = prob.solve_condensed(ru, rh)
    a, b = prob.integral_of_h(h), prob.integral_of_h(rh)
    assert abs(a - b) <= 1e-12 * prob.integral_of_h(np.abs(rh))


def _l2_error(prob, mesh, u, h, exact):
    xi, eta, w = triangle_rule(8)
    phi = ref.eval_cell_basis(prob.prm.p, xi, eta)
    X = mesh.cell_coords()
    eu = eh = 0.0
    for K in range(prob.N):
        detJ = cell_geometry(prob.X[K])[0]
        pts = X[K, 0] + np.outer(xi, X[K, 1] - X[K, 0]) + np.outer(eta, X[K, 2] - X[K, 0])
        ux, uy, hh = exact(pts)
        eu += detJ * w @ ((phi @ u[K, 0] - ux) ** 2 + (phi @ u[K, 1] - uy) ** 2)
        eh += detJ * w @ (phi @ h[K] - hh) ** 2
    return math.sqrt(eu), math.sqrt(eh)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_manufactured_convergence(p):
    """Sec. 7.3: L2 errors decrease at least like h^(p+1/2); p+1 is expected."""
    g, H, f0 = 1.0, 1.0, 1.0
    errs = []
    for n in (4, 8, 16):
        mesh = I.periodic_square(n)
        tau = 8 * mesh.h          # acoustic Courant number 8 (c = 1)
        prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=I.coriolis_flat(mesh, f0), tau_s=1.0)
        ru, rh = I.manufactured_rhs(mesh, p, tau, g, H, f0)
        (u, h), _ = prob.solve_condensed(ru, rh)
        errs.append(_l2_error(prob, mesh, u, h, lambda x: I.fields.manufactured_solution(x, 1.0, 1.0, 1.0)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates[-1] >= p + 0.5).all(), rates


@pytest.mark.parametrize("p", [2, 3, 4])
def test_fourier_closed_form(p):
    """Single Fourier mode on the periodic square with constant f: the
    continuous solution is a 3x3 complex solve per mode; the discrete error
    converges at order >= p + 1/2."""
    g, H, f0, tau = 1.0, 2.0, 0.7, 0.05
    kv = 2 * math.pi * np.array([1.0, 2.0])
    Mc = np.array([[1, -tau * f0, 1j * tau * g * kv[0]],
                   [tau * f0, 1, 1j * tau * g * kv[1]],
                   [1j * tau * H * kv[0], 1j * tau * H * kv[1], 1]], dtype=complex)
    sol = np.linalg.solve(Mc, np.array([0, 0, 1.0 + 0j]))   # r = (0, 0, e^{ik.x})

    def exact(x):
        ph = np.exp(1j * (x @ kv))
        return (sol[0] * ph).real, (sol[1] * ph).real, (sol[2] * ph).real

    errs = []
    for n in (4, 8, 16):
        mesh = I.periodic_square(n)
        prob = HDGProblem(mesh, p, tau=tau, g=g, H=H, f_vertex=I.coriolis_flat(mesh, f0))
        xy = I.dg_node_positions(mesh, p)
        rh = np.cos(xy @ kv)
        ru = np.zeros((mesh.n_cells, 2, prob.np))
        (u, h), _ = prob.solve_condensed(ru, rh)
        errs.append(_l2_error(prob, mesh, u, h, exact))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates[-1] >= p + 0.5).all(), rates


def _tau_limit_deviation(tau):
    mesh, prob = _problem("flat", 2, tau=tau)
    ru, rh = _rand_rhs(prob, 5)
    (u, h), lam = prob.solve_condensed(ru, rh)
    # upwind trace value from both sides at every trace node
    R = ref.reference_matrices(prob.prm.p)
    pp = prob.prm.p + 1
    acc = np.zeros(prob.n_trace)
    for K in range(prob.N):
        _, _, _, normals = cell_geometry(prob.X[K])
        for i in range(3):
            T = np.linalg.solve(R["M1"], R["N"][i].T)        # cell coeffs -> trace nodal values
            hv = T @ rh[K]
            un = T @ (normals[i][0] * ru[K, 0] + normals[i][1] * ru[K, 1])
            np.add.at(acc, prob.gdof[K, i * pp:(i + 1) * pp],
                      0.5 * hv + prob.prm.H / (2 * prob.prm.tau_s) * un)
    return np.array([np.abs(u - ru).max(), np.abs(h - rh).max(), np.abs(lam - acc).max()])


def test_tau_to_zero_limit():
    """tau -> 0: (u, h) -> (r_u, r_h) and lambda -> {h} + H/(2 tau_s) [[u]] (the
    upwind value), with a deviation that is O(tau)."""
    d1 = _tau_limit_deviation(1e-10)
    d2 = _tau_limit_deviation(1e-11)
    assert (d2 < 1e-8).all(), d2
    assert np.allclose(d1 / d2, 10.0, rtol=1e-3), d1 / d2


@pytest.mark.parametrize("kind", ["flat", "sphere"])
def test_p1_injection_is_the_trace(kind):
    """pi phi_c at each trace node equals the P1 function evaluated at that node."""
    mesh, prob = _problem(kind, 3)
    rng = np.random.default_rng(6)
    phic = rng.standard_normal(mesh.n_vertices)
    Pi = injection(prob, mesh.n_vertices).toarray()
    lam = Pi @ phic
    X = mesh.cell_coords()
    pp = prob.prm.p + 1
    for K in range(prob.N):
        vv = mesh.cell_vertices[K]
        for i in range(3):
            a, b = (i + 1) % 3, (i + 2) % 3
            for j in range(pp):
                t = j / prob.prm.p
                # P1 function along the edge, from local vertex a to b
                val = (1 - t) * phic[vv[a]] + t * phic[vv[b]]
                assert abs(lam[prob.gdof[K, i * pp + j]] - val) < 1e-13


def test_dof_counts_match_paper_tables():
    with open(os.path.join(GOLDEN, "dof_counts.json")) as fh:
        tab = json.load(fh)
    from oracle.hdg import facet_numbering
    for row in tab["flat"]:
        n = 2 ** row["r"]
        mesh = I.periodic_square(n)
        assert mesh.n_cells == row["n_cell"]
        nf = facet_numbering(mesh.cell_vertices)[2].shape[0]
        for p, (ncell, nfacet) in row["p"].items():
            p = int(p)
            assert 3 * (p + 1) * (p + 2) // 2 * mesh.n_cells == ncell
            assert (p + 1) * nf == nfacet
    for row in tab["sphere"]:
        if row["r"] > 6:
            continue     # r = 7 takes long in pure Python; r <= 6 covers the formula
        mesh = I.icosahedral_sphere(row["r"])
        assert mesh.n_cells == row["n_cell"]
        assert abs(mesh.h - row["h"]) < 1e-4
        nf = facet_numbering(mesh.cell_vertices)[2].shape[0]
        for p, (ncell, nfacet) in row["p"].items():
            p = int(p)
            assert 3 * (p + 1) * (p + 2) // 2 * mesh.n_cells == ncell
            assert (p + 1) * nf == nfacet
