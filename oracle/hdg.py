"""HDG discretisation of the implicit linear rotating shallow-water step (oracle).

Test infrastructure only (see the package docstring).

The system solved (the upwind HDG form of Eq. bilinear_HDG_upwind written with
tau = alpha*Delta t, the paper's c_g*phi_B -> g, c_g -> H, c_g*sqrt(phi_B) ->
tau_s = sqrt(g H), phi -> h, phi_hat -> lambda, plus the Coriolis term taken
implicitly), for every cell K and all test functions w, psi, mu:

    (u,w)_K + tau (f u_perp, w)_K - tau g (h, div w)_K + tau g <lambda, w.n>_dK = (r_u, w)_K
    (h,psi)_K - tau H (u, grad psi)_K + tau <H u.n + tau_s (h - lambda), psi>_dK = (r_h, psi)_K
    sum_{K containing e} <H u.n_K + tau_s (h - lambda), mu>_e = 0          (every facet e)

u_perp = (-u_y, u_x).  The last line is the weak flux continuity of
Eq. flux_condition, scaled by c_g.  In the ABCM notation of Eq. ABCMform
(App. B, upwind) the cell rows are ``A_K q + B_K lambda = F_K`` and the facet
rows ``sum_K (C_K q_K - Mt_K lambda) = 0`` with ``Mt_K = tau_s M_dK``.

Geometry: flat cells use their (periodic-unwrapped) Cartesian vertices; cells
of the sphere mesh are flat triangles written in their own frame
``e1 = (X1-X0)/|X1-X0|, e2 = n x e1``, so every cell is handled as a 2-D cell
and only the scalar trace couples cells.

Numbering (shared convention, computed here independently of the library):
facet ids in order of first appearance over (cell, local edge); the trace
nodes of a facet run from its lower global vertex id to the higher.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import reference as ref


# ------------------------------------------------------------------ mesh data

@dataclass
class MeshData:
    dim: int
    vertex_xyz: np.ndarray
    cell_vertices: np.ndarray
    cell_shift: np.ndarray | None

    @classmethod
    def of(cls, mesh) -> "MeshData":
        return cls(mesh.dim, np.asarray(mesh.vertex_xyz, np.float64),
                   np.asarray(mesh.cell_vertices, np.int64),
                   None if mesh.cell_shift is None else np.asarray(mesh.cell_shift, np.float64))

    @property
    def n_cells(self) -> int:
        return self.cell_vertices.shape[0]


def facet_numbering(cell_vertices: np.ndarray):
    """Return (facet_of [N,3], flip [N,3] bool, facet_verts [nf,2] (lo, hi)).

    Local edge i joins local vertices (i+1)%3 -> (i+2)%3; ``flip`` is True
    when that direction runs from the higher to the lower global vertex id.
    Raises ValueError unless every facet has exactly two incident cells.
    """
    N = cell_vertices.shape[0]
    facet_of = np.empty((N, 3), dtype=np.int64)
    flip = np.empty((N, 3), dtype=bool)
    ids: dict[tuple[int, int], int] = {}
    count: list[int] = []
    verts: list[tuple[int, int]] = []
    for K in range(N):
        for i in range(3):
            a = int(cell_vertices[K, (i + 1) % 3])
            b = int(cell_vertices[K, (i + 2) % 3])
            key = (min(a, b), max(a, b))
            if key not in ids:
                ids[key] = len(verts)
                verts.append(key)
                count.append(0)
            e = ids[key]
            count[e] += 1
            facet_of[K, i] = e
            flip[K, i] = a > b
    if any(c != 2 for c in count):
        raise ValueError("mesh is not a closed 2-manifold: a facet does not have two cells")
    return facet_of, flip, np.array(verts, dtype=np.int64)


def local_coordinates(md: MeshData) -> np.ndarray:
    """2-D vertex coordinates of every cell, float64 [N, 3, 2]."""
    x = md.vertex_xyz[md.cell_vertices]
    if md.cell_shift is not None:
        x = x + md.cell_shift
    if md.dim == 2:
        return x.copy()
    out = np.empty((x.shape[0], 3, 2))
    for K in range(x.shape[0]):
        d1 = x[K, 1] - x[K, 0]
        d2 = x[K, 2] - x[K, 0]
        e1 = d1 / np.linalg.norm(d1)
        nrm = np.cross(d1, d2)
        nrm /= np.linalg.norm(nrm)
        e2 = np.cross(nrm, e1)
        for v in range(3):
            d = x[K, v] - x[K, 0]
            out[K, v] = (d @ e1, d @ e2)
    return out


# ------------------------------------------------------------------ local operators

@dataclass
class Params:
    p: int
    tau: float
    g: float
    H: float
    tau_s: float


def cell_geometry(X: np.ndarray):
    """detJ, inverse-transpose Jacobian, edge lengths and outward unit normals."""
    J = np.array([[X[1, 0] - X[0, 0], X[2, 0] - X[0, 0]],
                  [X[1, 1] - X[0, 1], X[2, 1] - X[0, 1]]])
    detJ = np.linalg.det(J)
    if detJ <= 0:
        raise ValueError("cell is not counter-clockwise")
    Jit = np.linalg.inv(J).T
    lengths = np.empty(3)
    normals = np.empty((3, 2))
    for i in range(3):
        t = X[(i + 2) % 3] - X[(i + 1) % 3]
        lengths[i] = np.linalg.norm(t)
        normals[i] = (t[1] / lengths[i], -t[0] / lengths[i])
    return detJ, Jit, lengths, normals


def local_operators(X: np.ndarray, f_cell: np.ndarray, prm: Params):
    """Cell matrices (A_K, B_K, C_K, Mt_K, Mass_K) of the form in the module
    docstring.  Unknown order within the cell: u_x nodes, u_y nodes, h nodes;
    local trace dofs: edge i, node j (in the edge's local direction) at
    ``i*(p+1) + j``."""
    p, tau, g, H, ts = prm.p, prm.tau, prm.g, prm.H, prm.tau_s
    R = ref.reference_matrices(p)
    n = R["n"]
    pp = p + 1
    detJ, Jit, lengths, normals = cell_geometry(X)
    M = detJ * R["M"]
    Mf = detJ * sum(f_cell[i] * R["ML"][i] for i in range(3))
    # Dx[a,b] = int phi_a d_x phi_b, Dy likewise
    Dx = detJ * (Jit[0, 0] * R["Dxi"] + Jit[0, 1] * R["Deta"])
    Dy = detJ * (Jit[1, 0] * R["Dxi"] + Jit[1, 1] * R["Deta"])
    ux, uy, hh = slice(0, n), slice(n, 2 * n), slice(2 * n, 3 * n)

    A = np.zeros((3 * n, 3 * n))
    # momentum, test w = phi_a e_x / phi_a e_y
    A[ux, ux] += M
    A[uy, uy] += M
    A[ux, uy] += -tau * Mf          # f u_perp . e_x = -f u_y
    A[uy, ux] += tau * Mf           # f u_perp . e_y = +f u_x
    A[ux, hh] += -tau * g * Dx.T    # -tau g (h, d_x phi_a)
    A[uy, hh] += -tau * g * Dy.T
    # mass, test psi = phi_a: volume term -tau H (u, grad psi)
    A[hh, hh] += M
    A[hh, ux] += -tau * H * Dx.T
    A[hh, uy] += -tau * H * Dy.T
    B = np.zeros((3 * n, 3 * pp))
    C = np.zeros((3 * pp, 3 * n))
    Mt = np.zeros((3 * pp, 3 * pp))
    for i in range(3):
        le, (nx, ny) = lengths[i], normals[i]
        E = le * R["E"][i]
        Nn = le * R["N"][i]
        sl = slice(i * pp, (i + 1) * pp)
        # mass row boundary terms: tau <H u.n + tau_s h, psi>
        A[hh, ux] += tau * H * nx * E
        A[hh, uy] += tau * H * ny * E
        A[hh, hh] += tau * ts * E
        # lambda couplings: tau g <lambda, w.n>, -tau tau_s <lambda, psi>
        B[ux, sl] += tau * g * nx * Nn
        B[uy, sl] += tau * g * ny * Nn
        B[hh, sl] += -tau * ts * Nn
        # transmission row: <H u.n + tau_s h, mu> - tau_s <lambda, mu>
        C[sl, ux] += H * nx * Nn.T
        C[sl, uy] += H * ny * Nn.T
        C[sl, hh] += ts * Nn.T
        Mt[sl, sl] += ts * le * R["M1"]
    Mass = np.zeros((3 * n, 3 * n))
    Mass[ux, ux] = M
    Mass[uy, uy] = M
    Mass[hh, hh] = M
    return A, B, C, Mt, Mass


def trace_dof_map(facet_of: np.ndarray, flip: np.ndarray, p: int) -> np.ndarray:
    """Global trace dof of every local trace dof, int64 [N, 3(p+1)]."""
    N = facet_of.shape[0]
    pp = p + 1
    out = np.empty((N, 3 * pp), dtype=np.int64)
    for K in range(N):
        for i in range(3):
            for j in range(pp):
                jj = p - j if flip[K, i] else j
                out[K, i * pp + j] = facet_of[K, i] * pp + jj
    return out


# ------------------------------------------------------------------ the discrete problem

class HDGProblem:
    """All cell operators of one mesh / parameter set, plus the assembled
    monolithic and condensed systems."""

    def __init__(self, mesh, p: int, tau: float, g: float, H: float,
                 f_vertex: np.ndarray, tau_s: float | None = None, lazy: bool = False):
        self.md = MeshData.of(mesh)
        self.prm = Params(p, tau, g, H, np.sqrt(g * H) if tau_s is None else tau_s)
        self.f_vertex = np.asarray(f_vertex, np.float64)
        self.facet_of, self.flip, self.facet_verts = facet_numbering(self.md.cell_vertices)
        self.n_facets = self.facet_verts.shape[0]
        self.X = local_coordinates(self.md)
        self.N = self.md.n_cells
        self.np = ref.n_cell_nodes(p)
        self.nK = 3 * self.np
        self.m = 3 * (p + 1)
        self.n_trace = self.n_facets * (p + 1)
        self.gdof = trace_dof_map(self.facet_of, self.flip, p)
        # cell operators, built on first use when lazy (large meshes checked on samples)
        self._ops: dict[int, tuple] = {}
        if not lazy:
            for K in range(self.N):
                self.op(K)

    def op(self, K: int):
        """(A_K, B_K, C_K, Mt_K, Mass_K) of cell K."""
        K = int(K)
        if K not in self._ops:
            fK = self.f_vertex[self.md.cell_vertices[K]]
            self._ops[K] = local_operators(self.X[K], fK, self.prm)
        return self._ops[K]

    @property
    def ops(self):
        return [self.op(K) for K in range(self.N)]

    # -- input layout helpers
    def cell_rhs(self, r_u: np.ndarray, r_h: np.ndarray) -> np.ndarray:
        """Per-cell nodal RHS vectors [N, nK] in the local unknown order."""
        return np.concatenate([r_u[:, 0, :], r_u[:, 1, :], r_h], axis=1)

    def load(self, r_u, r_h) -> np.ndarray:
        """F_K = Mass_K r_K (the Riesz map of the RHS functions)."""
        rc = self.cell_rhs(r_u, r_h)
        return np.stack([self.op(K)[4] @ rc[K] for K in range(self.N)])

    def local_cells(self, cells, r_u, r_h, lam):
        """Step 3 for selected cells only: q_K = A_K^-1 (Mass_K r_K - B_K lambda_K)."""
        out = []
        for K in cells:
            A, B, C, Mt, Mass = self.op(K)
            rK = np.concatenate([r_u[K, 0], r_u[K, 1], r_h[K]])
            out.append(np.linalg.solve(A, Mass @ rK - B @ lam[self.gdof[K]]))
        return np.array(out)

    def facet_rows(self, facets, x):
        """(S x) restricted to the trace dofs of the selected facets, from the
        S_K of their two cells."""
        pp = self.prm.p + 1
        cells_of = {}
        for K in range(self.N):
            for i in range(3):
                cells_of.setdefault(int(self.facet_of[K, i]), []).append(K)
        out = []
        for e in facets:
            y = np.zeros(self.n_trace)
            for K in cells_of[int(e)]:
                np.add.at(y, self.gdof[K], self.cell_schur(K) @ x[self.gdof[K]])
            out.append(y[int(e) * pp:(int(e) + 1) * pp])
        return np.array(out)

    def facet_rhs(self, facets, r_u, r_h):
        """Step 1 restricted to the selected facets."""
        pp = self.prm.p + 1
        cells_of = {}
        for K in range(self.N):
            for i in range(3):
                cells_of.setdefault(int(self.facet_of[K, i]), []).append(K)
        out = []
        for e in facets:
            gl = np.zeros(self.n_trace)
            for K in cells_of[int(e)]:
                A, B, C, Mt, Mass = self.op(K)
                rK = np.concatenate([r_u[K, 0], r_u[K, 1], r_h[K]])
                np.add.at(gl, self.gdof[K], C @ np.linalg.solve(A, Mass @ rK))
            out.append(gl[int(e) * pp:(int(e) + 1) * pp])
        return np.array(out)

    # -- route (i): the monolithic system
    def monolithic(self):
        nK, m, N = self.nK, self.m, self.N
        nq = N * nK
        rows, cols, vals = [], [], []
        for K in range(N):
            A, B, C, Mt, _ = self.op(K)
            q0 = K * nK
            qi = q0 + np.arange(nK)
            li = nq + self.gdof[K]
            for (blk, r, c) in ((A, qi, qi), (B, qi, li), (C, li, qi), (-Mt, li, li)):
                rr, cc = np.meshgrid(r, c, indexing="ij")
                rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(blk.ravel())
        n = nq + self.n_trace
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n))

    def solve_monolithic(self, r_u, r_h):
        Amono = self.monolithic()
        F = self.load(r_u, r_h)
        rhs = np.concatenate([F.ravel(), np.zeros(self.n_trace)])
        sol = spla.splu(Amono.tocsc()).solve(rhs)
        q = sol[: self.N * self.nK].reshape(self.N, self.nK)
        return self.split(q), sol[self.N * self.nK:]

    def split(self, q: np.ndarray):
        n = self.np
        u = np.stack([q[:, 0:n], q[:, n:2 * n]], axis=1)
        return u, q[:, 2 * n:3 * n]

    # -- route (ii): Schur complement (Sec. 4.2, steps 1-3)
    def cell_schur(self, K: int) -> np.ndarray:
        """S_K = Mt_K + C_K A_K^-1 B_K (local trace order)."""
        A, B, C, Mt, _ = self.op(K)
        return Mt + C @ np.linalg.solve(A, B)

    def trace_operator(self) -> sp.csr_matrix:
        """S+ = sum_K P_K^T (Mt_K + C_K A_K^-1 B_K) P_K (Eq. schur_system)."""
        rows, cols, vals = [], [], []
        for K in range(self.N):
            SK = self.cell_schur(K)
            rr, cc = np.meshgrid(self.gdof[K], self.gdof[K], indexing="ij")
            rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(SK.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_trace, self.n_trace))

    def condensed_rhs(self, r_u, r_h) -> np.ndarray:
        """Step 1: g = sum_K P_K^T C_K A_K^-1 F_K."""
        F = self.load(r_u, r_h)
        gvec = np.zeros(self.n_trace)
        for K in range(self.N):
            A, B, C, Mt, _ = self.op(K)
            np.add.at(gvec, self.gdof[K], C @ np.linalg.solve(A, F[K]))
        return gvec

    def recover(self, lam: np.ndarray, r_u, r_h):
        """Step 3: q_K = A_K^-1 (F_K - B_K lambda_K) (Eq. reconstruct_solution)."""
        F = self.load(r_u, r_h)
        q = np.empty((self.N, self.nK))
        for K in range(self.N):
            A, B, C, Mt, _ = self.op(K)
            q[K] = np.linalg.solve(A, F[K] - B @ lam[self.gdof[K]])
        return self.split(q)

    def solve_condensed(self, r_u, r_h):
        S = self.trace_operator()
        gvec = self.condensed_rhs(r_u, r_h)
        lam = spla.splu(S.tocsc()).solve(gvec)
        return self.recover(lam, r_u, r_h), lam

    # -- quantities used by the pins
    def cell_mass(self, K: int) -> np.ndarray:
        return self.op(K)[4][2 * self.np:, 2 * self.np:]

    def integral_of_h(self, h: np.ndarray) -> float:
        R = ref.reference_matrices(self.prm.p)
        w = R["M"].sum(axis=0)          # int phi_b over the reference cell
        return float(sum(cell_geometry(self.X[K])[0] * w @ h[K] for K in range(self.N)))

    def l2_norm2_cells(self, v: np.ndarray) -> float:
        """sum_K v_K^T M_K v_K for a scalar DG field v [N, n_p]."""
        return float(sum(v[K] @ self.cell_mass(K) @ v[K] for K in range(self.N)))

    def facet_dof_positions(self) -> np.ndarray:
        """Parameter t in [0,1] from the lower to the higher vertex of each trace node."""
        return np.arange(self.prm.p + 1) / self.prm.p


def dense(S) -> np.ndarray:
    return S.toarray() if sp.issparse(S) else np.asarray(S)


def lu_solve_dense(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    return sla.lu_solve(sla.lu_factor(A), b)
