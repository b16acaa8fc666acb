"""Standard (non-hybridised) upwind DG system in (u, h) only (oracle cross-check).

Test infrastructure only (see the package docstring).

The paper states that the HDG solution q equals the solution of the
non-hybridised DG discretisation (the remark after Eq. linear_hybridized).
Here that equivalence is used as an independent route: every facet is
straight and every trace lies in P^p(e), so the facet equation of the HDG
system holds pointwise and gives

    lambda = {h} + (H / (2 tau_s)) (u_K1 . n_K1 + u_K2 . n_K2)   on each facet,

which is substituted into the cell equations.  The cell terms are written
in the integrated-by-parts form of the mass equation,

    (h,psi)_K + tau H (div u, psi)_K + tau tau_s <h - lambda, psi>_dK = (r_h, psi)_K,

(different arithmetic from the HDG assembly, which keeps
-tau H (u, grad psi) + tau H <u.n, psi>), so that agreement checks both.
Neighbour traces are evaluated by running the shared edge in the opposite
direction (both cells are counter-clockwise).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import reference as ref
from .hdg import HDGProblem, cell_geometry


def _cross_edge_matrix(p: int, i: int, i2: int) -> np.ndarray:
    """X[a,b] = int_0^1 phi_a(edge i at t) phi_b(edge i2 at 1-t) dt."""
    phi = ref.cell_basis(p)
    A, B = ref.edge_endpoints(i)
    A2, B2 = ref.edge_endpoints(i2)
    own = [ref.on_segment(c, A, B) for c in phi]
    nbr = [ref.on_segment(c, B2, A2) for c in phi]      # reversed direction
    n = len(phi)
    return np.array([[float(ref.integrate_unit(ref.mul1(own[a], nbr[b]))) for b in range(n)]
                     for a in range(n)], dtype=np.float64)


def solve_standard_dg(prob: HDGProblem, r_u: np.ndarray, r_h: np.ndarray):
    """Assemble and solve the standard upwind DG system; returns (u, h)."""
    Amat = assemble_standard_dg(prob)
    rhs = prob.load(r_u, r_h).ravel()
    q = spla.splu(Amat.tocsc()).solve(rhs).reshape(prob.N, -1)
    return prob.split(q)


def assemble_standard_dg(prob: HDGProblem) -> sp.csr_matrix:
    """The matrix of the standard upwind DG system (cell unknowns ordered
    cell, then u_x, u_y, h, then node), so that A q = M r."""
    p = prob.prm.p
    tau, g, H, ts = prob.prm.tau, prob.prm.g, prob.prm.H, prob.prm.tau_s
    R = ref.reference_matrices(p)
    n = R["n"]
    N = prob.N
    nK = 3 * n
    # neighbour of (K, i)
    owner: dict[int, list[tuple[int, int]]] = {}
    for K in range(N):
        for i in range(3):
            owner.setdefault(int(prob.facet_of[K, i]), []).append((K, i))
    cross = {(i, i2): _cross_edge_matrix(p, i, i2) for i in range(3) for i2 in range(3)}

    rows, cols, vals = [], [], []

    def put(blk, K1, s1, K2, s2):
        r = K1 * nK + s1 * n + np.arange(n)
        c = K2 * nK + s2 * n + np.arange(n)
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(blk.ravel())

    geo = [cell_geometry(prob.X[K]) for K in range(N)]
    for K in range(N):
        detJ, Jit, lengths, normals = geo[K]
        fK = prob.f_vertex[prob.md.cell_vertices[K]]
        M = detJ * R["M"]
        Mf = detJ * sum(fK[i] * R["ML"][i] for i in range(3))
        Dx = detJ * (Jit[0, 0] * R["Dxi"] + Jit[0, 1] * R["Deta"])
        Dy = detJ * (Jit[1, 0] * R["Dxi"] + Jit[1, 1] * R["Deta"])
        UX, UY, HH = 0, 1, 2
        put(M, K, UX, K, UX)
        put(M, K, UY, K, UY)
        put(-tau * Mf, K, UX, K, UY)
        put(tau * Mf, K, UY, K, UX)
        put(-tau * g * Dx.T, K, UX, K, HH)
        put(-tau * g * Dy.T, K, UY, K, HH)
        put(M, K, HH, K, HH)
        put(tau * H * Dx, K, HH, K, UX)      # tau H (d_x u_x, psi_a)
        put(tau * H * Dy, K, HH, K, UY)
        for i in range(3):
            le, (nx, ny) = lengths[i], normals[i]
            E = le * R["E"][i]
            put(tau * ts * E, K, HH, K, HH)
            (K2, i2), = [oi for oi in owner[int(prob.facet_of[K, i])] if oi != (K, i)]
            Xc = le * cross[(i, i2)]
            n2x, n2y = geo[K2][3][i2]
            # lambda = 0.5 (h_K + h_K2) + H/(2 tau_s) (u_K.n_K + u_K2.n_K2)
            lam_terms = [
                (K, HH, 0.5 * E), (K, UX, H / (2 * ts) * nx * E), (K, UY, H / (2 * ts) * ny * E),
                (K2, HH, 0.5 * Xc), (K2, UX, H / (2 * ts) * n2x * Xc), (K2, UY, H / (2 * ts) * n2y * Xc),
            ]
            for (Kc, sc, blk) in lam_terms:
                put(tau * g * nx * blk, K, UX, Kc, sc)     # tau g <lambda, w.n>
                put(tau * g * ny * blk, K, UY, Kc, sc)
                put(-tau * ts * blk, K, HH, Kc, sc)        # -tau tau_s <lambda, psi>
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N * nK, N * nK))
