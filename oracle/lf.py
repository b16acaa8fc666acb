"""Lax-Friedrichs HDG variant with a vector trace and the RT0 coarse space (oracle).

Test infrastructure only (see the package docstring).

The Lax-Friedrichs form of Eq. bilinear_HDG_lax, with the dictionary of the
upwind oracle (tau = alpha*Delta t, c_g*phi_B -> g, c_g -> H,
c_g*sqrt(phi_B) -> tau_s = sqrt(g H)) and the Coriolis term implicit, couples
cell fields (u, h) to a *vector* trace u_hat in [P^p(e)]^2 on every facet;
the height has no trace (the form does not depend on phi_hat).  Per cell K and
test functions w, psi, and per facet e and test w_hat:

    (u,w)_K + tau f (u_perp,w)_K - tau g (h, div w)_K + tau g <h, w.n>_dK
        + tau tau_s <u - u_hat, w>_dK                             = (r_u, w)_K
    (h,psi)_K - tau H (u, grad psi)_K + tau H <u_hat.n, psi>_dK   = (r_h, psi)_K
    sum_{K containing e} <g h_K n_K + tau_s (u_K - u_hat), w_hat>_e = 0

(the facet terms of Eq. bilinear_HDG_lax written cell by cell: 2 sqrt(phi_B)
({u.w} - u_hat.{w}) and phi_B [[phi w]] give the stabilisation and the
own-side height flux; the last line is the transmission condition of the
form's w_hat term, scaled by c_g).  In the ABCM split (App. B) the cell rows
are A_K q + B_K u_hat = F_K and the facet rows sum_K (C_K q_K - Mt_K u_hat) = 0
with Mt_K = tau_s M_dK per component; the trace system is again
S+ u_hat = sum_K C_K A_K^-1 F_K with S+ = sum_K (Mt_K + C_K A_K^-1 B_K).

Flat periodic meshes only: the trace components are Cartesian (on the folded
sphere the two cells of a facet have different tangent planes and the vector
trace would need a facet frame).  Trace dofs of facet e: component c (x, y),
node j from the lower to the higher vertex id, at e*2(p+1) + c*(p+1) + j.

Coarse space (Sec. 4.4, Lax-Friedrichs): the lowest-order Raviart-Thomas
space RT0, one normal-flux dof per facet (sign fixed by the facet's global
normal nu_e, the edge direction lo -> hi turned clockwise).  Prolongation pi:
u_hat = the L2 projection on the skeleton of the average {u_c} of the two
cells' RT0 fields; RT0 fields are linear along a facet, so the projection
onto P^p(e) (p >= 1) is nodal interpolation.  Coarse operator
(Eq. coarse_problem_LF with the implicit Coriolis term added the way the
upwind coarse problem adds it): the grad-div form
    S_c(u_c, w_c) = (u_c, w_c) + tau f (u_c_perp, w_c) + tau^2 g H (div u_c, div w_c),
divided by tau, the scale at which S+ acts on smooth traces: testing the cell
rows with (u, (g/H) h) and the transmission rows with u_hat gives the energy
identity
    u_hat^T S+ u_hat = (1/tau)(||u||^2 + (g/H)||h||^2) + tau_s sum_K ||u - u_hat||^2_dK
for the local responses (u, h) to u_hat (f = 0, zero right-hand side), and
h = -tau H div u for smooth fields; or the Galerkin product pi^T S+ pi of the
Sec. 4.4 footnote.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import reference as ref
from .hdg import HDGProblem, Params, cell_geometry


def local_operators_lf(X: np.ndarray, f_cell: np.ndarray, prm: Params):
    """(A_K, B_K, C_K, Mt_K, Mass_K) of the Lax-Friedrichs form above.  Cell
    unknowns u_x, u_y, h (nodes each); local trace dofs: edge i, component c,
    node j (in the edge's local direction) at i*2(p+1) + c*(p+1) + j."""
    p, tau, g, H, ts = prm.p, prm.tau, prm.g, prm.H, prm.tau_s
    R = ref.reference_matrices(p)
    n = R["n"]
    pp = p + 1
    detJ, Jit, lengths, normals = cell_geometry(X)
    M = detJ * R["M"]
    Mf = detJ * sum(f_cell[i] * R["ML"][i] for i in range(3))
    Dx = detJ * (Jit[0, 0] * R["Dxi"] + Jit[0, 1] * R["Deta"])   # Dx[a,b] = int phi_a d_x phi_b
    Dy = detJ * (Jit[1, 0] * R["Dxi"] + Jit[1, 1] * R["Deta"])
    ux, uy, hh = slice(0, n), slice(n, 2 * n), slice(2 * n, 3 * n)
    comp = (ux, uy)
    A = np.zeros((3 * n, 3 * n))
    A[ux, ux] += M
    A[uy, uy] += M
    A[ux, uy] += -tau * Mf                  # f u_perp . e_x = -f u_y
    A[uy, ux] += tau * Mf
    A[ux, hh] += -tau * g * Dx.T            # -tau g (h, d_x phi_a)
    A[uy, hh] += -tau * g * Dy.T
    A[hh, hh] += M
    A[hh, ux] += -tau * H * Dx.T            # -tau H (u, grad psi)
    A[hh, uy] += -tau * H * Dy.T
    B = np.zeros((3 * n, 6 * pp))
    C = np.zeros((6 * pp, 3 * n))
    Mt = np.zeros((6 * pp, 6 * pp))
    for i in range(3):
        le, nrm = lengths[i], normals[i]
        E = le * R["E"][i]
        Nn = le * R["N"][i]
        for c in range(2):
            sl = slice(i * 2 * pp + c * pp, i * 2 * pp + (c + 1) * pp)
            # momentum: tau g <h, w.n> (own-side height) and tau tau_s <u - u_hat, w>
            A[comp[c], hh] += tau * g * nrm[c] * E
            A[comp[c], comp[c]] += tau * ts * E
            B[comp[c], sl] += -tau * ts * Nn
            # mass: tau H <u_hat.n, psi>
            B[hh, sl] += tau * H * nrm[c] * Nn
            # transmission, component c: <g h n_c + tau_s u_c, mu> - tau_s <u_hat_c, mu>
            C[sl, hh] += g * nrm[c] * Nn.T
            C[sl, comp[c]] += ts * Nn.T
            Mt[sl, sl] += ts * le * R["M1"]
    Mass = np.zeros((3 * n, 3 * n))
    Mass[ux, ux] = M
    Mass[uy, uy] = M
    Mass[hh, hh] = M
    return A, B, C, Mt, Mass


def lf_trace_dof_map(facet_of: np.ndarray, flip: np.ndarray, p: int) -> np.ndarray:
    """Global trace dof of every local trace dof, int64 [N, 6(p+1)]."""
    N = facet_of.shape[0]
    pp = p + 1
    out = np.empty((N, 6 * pp), dtype=np.int64)
    for K in range(N):
        for i in range(3):
            for c in range(2):
                for j in range(pp):
                    jj = p - j if flip[K, i] else j
                    out[K, i * 2 * pp + c * pp + j] = facet_of[K, i] * 2 * pp + c * pp + jj
    return out


class LFProblem(HDGProblem):
    """The Lax-Friedrichs discretisation (flat meshes); the condensation,
    recovery and monolithic routes are those of HDGProblem on these operators."""

    def __init__(self, mesh, p: int, tau: float, g: float, H: float, f_vertex: np.ndarray,
                 tau_s: float | None = None, lazy: bool = False):
        if mesh.dim != 2:
            raise ValueError("the Lax-Friedrichs oracle handles flat (dim = 2) meshes")
        super().__init__(mesh, p, tau, g, H, f_vertex, tau_s=tau_s, lazy=True)
        self.m = 6 * (p + 1)
        self.n_trace = self.n_facets * 2 * (p + 1)
        self.gdof = lf_trace_dof_map(self.facet_of, self.flip, p)
        self._ops = {}
        if not lazy:
            for K in range(self.N):
                self.op(K)

    def op(self, K: int):
        K = int(K)
        if K not in self._ops:
            fK = self.f_vertex[self.md.cell_vertices[K]]
            self._ops[K] = local_operators_lf(self.X[K], fK, self.prm)
        return self._ops[K]


# ------------------------------------------------------------------ RT0 coarse space

def facet_normals(prob: LFProblem) -> np.ndarray:
    """Global unit normal nu_e of every facet: the direction lo -> hi turned
    clockwise, taken from the first cell's local coordinates (flat meshes)."""
    nu = np.empty((prob.n_facets, 2))
    done = np.zeros(prob.n_facets, dtype=bool)
    for K in range(prob.N):
        _, _, lengths, normals = cell_geometry(prob.X[K])
        for i in range(3):
            e = prob.facet_of[K, i]
            if done[e]:
                continue
            a, b = prob.X[K, (i + 1) % 3], prob.X[K, (i + 2) % 3]
            t = (b - a) if not prob.flip[K, i] else (a - b)       # lo -> hi
            t = t / np.linalg.norm(t)
            nu[e] = (t[1], -t[0])
            done[e] = True
    return nu


def rt0_cell_basis(X: np.ndarray, i: int, x: np.ndarray) -> np.ndarray:
    """RT0 basis function of local edge i of a cell at points x [k, 2]: unit
    outward normal component on edge i, zero normal component on the others:
    phi_i(x) = |e_i| / (2 |K|) (x - X_i)."""
    detJ, _, lengths, _ = cell_geometry(X)
    return lengths[i] / detJ * (x - X[i])          # |K| = detJ / 2


def rt0_injection(prob: LFProblem) -> sp.csr_matrix:
    """pi: RT0 dofs (normal flux per facet along nu_e) -> trace dofs, the
    average of the two cells' RT0 fields at the trace nodes."""
    p, pp = prob.prm.p, prob.prm.p + 1
    nu = facet_normals(prob)
    rows, cols, vals = [], [], []
    for K in range(prob.N):
        X = prob.X[K]
        _, _, _, normals = cell_geometry(X)
        sig = [1.0 if normals[i] @ nu[prob.facet_of[K, i]] > 0 else -1.0 for i in range(3)]
        for i in range(3):                                  # the facet whose trace is evaluated
            a, b = X[(i + 1) % 3], X[(i + 2) % 3]
            t = np.arange(pp) / p
            pts = a[None, :] + t[:, None] * (b - a)[None, :]   # edge-local node order
            for i2 in range(3):                             # RT0 dofs of the cell
                val = 0.5 * sig[i2] * rt0_cell_basis(X, i2, pts)     # [pp, 2]
                for c in range(2):
                    for j in range(pp):
                        rows.append(prob.gdof[K, i * 2 * pp + c * pp + j])
                        cols.append(prob.facet_of[K, i2])
                        vals.append(val[j, c])
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.n_trace, prob.n_facets))


def rt0_operator(prob: LFProblem, scale: float | None = None) -> sp.csr_matrix:
    """S_c = scale * [(u, w) + tau f (u_perp, w) + tau^2 g H (div u, div w)] on RT0
    (cell means of f; scale defaults to 1 / tau)."""
    tau, g, H = prob.prm.tau, prob.prm.g, prob.prm.H
    if scale is None:
        scale = 1.0 / tau
    nu = facet_normals(prob)
    # degree-2 exact rule on the reference triangle (edge midpoints)
    lam = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
    rows, cols, vals = [], [], []
    for K in range(prob.N):
        X = prob.X[K]
        detJ, _, lengths, normals = cell_geometry(X)
        area = 0.5 * detJ
        sig = np.array([1.0 if normals[i] @ nu[prob.facet_of[K, i]] > 0 else -1.0 for i in range(3)])
        pts = lam @ X
        phi = np.stack([sig[i] * rt0_cell_basis(X, i, pts) for i in range(3)])   # [3 basis, 3 pts, 2]
        Mloc = area / 3.0 * np.einsum("ikc,jkc->ij", phi, phi)
        perp = np.stack([-phi[..., 1], phi[..., 0]], axis=-1)                    # phi_perp
        fK = float(prob.f_vertex[prob.md.cell_vertices[K]].mean())
        Rloc = area / 3.0 * np.einsum("ikc,jkc->ij", phi, perp)                   # (phi_j_perp, phi_i) at [i, j]
        div = sig * lengths / area                                                 # div phi_i
        Dloc = area * np.outer(div, div)
        A = scale * (Mloc + tau * fK * Rloc + tau * tau * g * H * Dloc)
        f = prob.facet_of[K]
        rr, cc = np.meshgrid(f, f, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(A.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(prob.n_facets, prob.n_facets))


# ------------------------------------------------------------------ two-level preconditioner

def facet_blocks_inverse(S: sp.csr_matrix, nf: int, bs: int) -> sp.csr_matrix:
    """Block-diagonal inverse of the facet diagonal blocks (bs x bs) of S."""
    idx = np.arange(nf)[:, None] * bs + np.arange(bs)[None, :]
    D = np.asarray(S.tocsr()[np.repeat(idx, bs, axis=1).ravel(), np.tile(idx, (1, bs)).ravel()]).reshape(nf, bs, bs)
    return sp.bsr_matrix((np.linalg.inv(D), np.arange(nf), np.arange(nf + 1)), shape=S.shape).tocsr()


class LFTwoLevelPreconditioner:
    """Alg. twolevel_vcycle for the Lax-Friedrichs trace system: n_pre damped
    block-Jacobi sweeps on the facet blocks (2(p+1) x 2(p+1)), residual,
    restriction r_c = pi^T r to RT0, coarse solve, u_hat += pi e_c, n_post sweeps.
    The coarse problem S_c e_c = r_c is solved exactly (coarse="exact") or
    approximately by n_coarse steps of the Jacobi-preconditioned Chebyshev
    iteration on S_c from zero (coarse="chebyshev"; ellipse (theta, delta^2) of
    D_c^-1 S_c given or fitted to Arnoldi Ritz values, as for the smoother of
    the upwind solver)."""

    def __init__(self, prob: LFProblem, S: sp.csr_matrix, n_pre: int = 2, n_post: int = 2,
                 omega: float = 2.0 / 3.0, coarse: str = "exact", coarse_mode: str = "rediscretised",
                 n_coarse: int = 20, cheb_c: tuple | None = None, cheb_steps: int = 20):
        from .solver import arnoldi_ritz, chebyshev_ellipse, chebyshev_start_vector
        self.prob, self.S = prob, S
        self.n_pre, self.n_post, self.omega = n_pre, n_post, omega
        self.Dinv = facet_blocks_inverse(S, prob.n_facets, 2 * (prob.prm.p + 1))
        self.Pi = rt0_injection(prob)
        if coarse_mode == "rediscretised":
            self.Sc = rt0_operator(prob).tocsr()
        elif coarse_mode == "galerkin":
            self.Sc = (self.Pi.T @ S @ self.Pi).tocsr()
        else:
            raise ValueError(coarse_mode)
        self.coarse = coarse
        if coarse == "exact":
            self._lu = spla.splu(self.Sc.tocsc())
        elif coarse == "chebyshev":
            self.dc = 1.0 / self.Sc.diagonal()
            self.n_coarse = n_coarse
            if cheb_c is None:
                ritz = arnoldi_ritz(lambda v: self.dc * (self.Sc @ v), chebyshev_start_vector(prob.n_facets),
                                    cheb_steps)
                cheb_c = chebyshev_ellipse(ritz)
            self.cheb_c = (float(cheb_c[0]), float(cheb_c[1]))
        else:
            raise ValueError(coarse)

    def coarse_solve(self, rc: np.ndarray) -> np.ndarray:
        if self.coarse == "exact":
            return self._lu.solve(rc)
        theta, delta2 = self.cheb_c
        s_prev = 1.0 / theta
        d = s_prev * self.dc * rc
        x = d.copy()
        for _ in range(1, self.n_coarse):
            s = 1.0 / (2.0 * theta - delta2 * s_prev)
            d = delta2 * s * s_prev * d + 2.0 * s * self.dc * (rc - self.Sc @ x)
            x = x + d
            s_prev = s
        return x

    def smooth(self, b: np.ndarray, x: np.ndarray, n: int) -> np.ndarray:
        for _ in range(n):
            x = x + self.omega * (self.Dinv @ (b - self.S @ x))
        return x

    def __call__(self, b: np.ndarray) -> np.ndarray:
        x = self.smooth(b, np.zeros_like(b), self.n_pre)
        r = b - self.S @ x
        ec = self.coarse_solve(self.Pi.T @ r)
        x = x + self.Pi @ ec
        return self.smooth(b, x, self.n_post)
