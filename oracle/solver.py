"""Iterative trace solve of the oracle: (F)GMRES + non-nested two-level V-cycle.

Test infrastructure only (see the package docstring).

* ``gmres``: right-preconditioned flexible GMRES(m) (Saad's FGMRES: the
  preconditioned vectors z_j are kept, so a preconditioner that changes from
  one call to the next is allowed), modified Gram-Schmidt Arnoldi, Givens
  rotations, stop on the *true* relative residual ``||b - A x|| / ||b||``.
* ``TwoLevelPreconditioner``: Alg. twolevel_vcycle with initial guess zero:
  n_pre damped block-Jacobi sweeps on the facet blocks (or n_pre steps of the
  block-Jacobi-preconditioned Chebyshev iteration, "chebyshev"), residual, restriction
  ``r_c = pi^T r`` (pi = the natural injection of P1 into the trace space,
  Sec. 4.4, upwind), coarse solve, ``x += pi e_c``, n_post sweeps.
* Coarse problem: the weak form of the second-order problem that the
  time-implicit continuum equations give after eliminating u (the recipe of
  Sec. 4.4, Eq. coarse_problem_upwind), divided by tau (the scale at which the
  trace operator acts on smooth traces, from the energy identity
  ``x^T S+ x = (1/tau)(||h||^2 + (H/g)||u||^2) + ...``).  With the Coriolis
  term implicit, u = (I - tau f J)(r_u - tau g grad h) / (1 + tau^2 f^2)
  (J the rotation by 90 degrees), so per cell K with f_K the mean of f:
      S_c(phi, psi) = (phi, psi) + tau^2 g H kappa_K [(grad phi, grad psi)_K
                                                     - tau f_K (J grad phi, grad psi)_K],
      kappa_K = 1 / (1 + tau^2 f_K^2)                      ("rotating", default)
  which is exactly Eq. coarse_problem_upwind when f = 0; or the paper's form
  without rotation ("rediscretised"); or the Galerkin choice pi^T S+ pi of
  the footnote in Sec. 4.4 ("galerkin").  It is
  solved exactly (sparse LU) or by a geometric P1 V-cycle over the nested
  coarse meshes (damped Jacobi smoothing, rediscretised level operators,
  sparse LU on the coarsest level).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hdg import HDGProblem, MeshData, local_coordinates, cell_geometry


# ------------------------------------------------------------------ GMRES

def gmres(apply_A, b: np.ndarray, precond=None, restart: int = 30, rtol: float = 1e-8,
          maxiter: int = 1000, x0: np.ndarray | None = None):
    """Return (x, info) with info = {iters, true_rel_res, converged, history}."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    M = (lambda v: v) if precond is None else precond
    bnorm = np.linalg.norm(b)
    history = []
    if bnorm == 0.0:
        return x, dict(iters=0, true_rel_res=0.0, converged=True, history=history)
    iters = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= rtol or iters >= maxiter:
            return x, dict(iters=iters, true_rel_res=rel, converged=rel <= rtol, history=history)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        s = np.zeros(restart + 1)
        s[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = M(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            s[j + 1] = -sn[j] * s[j]
            s[j] = cs[j] * s[j]
            iters += 1
            k = j + 1
            history.append(abs(s[j + 1]) / bnorm)
            if abs(s[j + 1]) / bnorm <= rtol or iters >= maxiter or Hm[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(Hm[:k, :k]), s[:k])
        x = x + Z[:k].T @ y


# ------------------------------------------------------------------ P1 spaces

def p1_rotating_operator(md: MeshData, f_vertex: np.ndarray, tau: float, g: float, H: float) -> sp.csr_matrix:
    """Coarse operator with implicit rotation (module docstring), divided by tau."""
    X = local_coordinates(md)
    nv = md.vertex_xyz.shape[0]
    gref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    Jrot = np.array([[0.0, -1.0], [1.0, 0.0]])          # u_perp = J u
    rows, cols, vals = [], [], []
    for K in range(md.n_cells):
        detJ, Jit, _, _ = cell_geometry(X[K])
        G = gref @ Jit.T                                 # row a = grad L_a
        fK = f_vertex[md.cell_vertices[K]].mean()
        kap = 1.0 / (1.0 + (tau * fK) ** 2)
        Me = detJ / 24.0 * (np.ones((3, 3)) + np.eye(3))
        Ke = 0.5 * detJ * G @ G.T                       # (grad L_b, grad L_a) at [a, b]
        Se = 0.5 * detJ * G @ (G @ Jrot.T).T            # (J grad L_b, grad L_a) at [a, b]
        Ae = (Me + tau * tau * g * H * kap * (Ke - tau * fK * Se)) / tau
        vv = md.cell_vertices[K]
        rr, cc = np.meshgrid(vv, vv, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(Ae.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nv, nv))


def coarse_vertex_values(fine_values: np.ndarray, parent: np.ndarray, n_coarse: int) -> np.ndarray:
    """Values at the vertices of a coarser level, taken from the finer-level
    vertex that coincides with each (parent pair (a, a))."""
    out = np.empty(n_coarse)
    for i, (a, b) in enumerate(parent):
        if a == b:
            out[a] = fine_values[i]
    return out


def p1_matrices(md: MeshData):
    """Assembled P1 mass and stiffness matrices on a (flat or sphere) mesh."""
    X = local_coordinates(md)
    nv = md.vertex_xyz.shape[0]
    gref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    rows, cols, mv, kv = [], [], [], []
    for K in range(md.n_cells):
        detJ, Jit, _, _ = cell_geometry(X[K])
        Me = detJ / 24.0 * (np.ones((3, 3)) + np.eye(3))
        G = gref @ Jit.T                 # row a = grad L_a
        Ke = 0.5 * detJ * G @ G.T
        vv = md.cell_vertices[K]
        rr, cc = np.meshgrid(vv, vv, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel())
        mv.append(Me.ravel()); kv.append(Ke.ravel())
    r, c = np.concatenate(rows), np.concatenate(cols)
    Mm = sp.csr_matrix((np.concatenate(mv), (r, c)), shape=(nv, nv))
    Km = sp.csr_matrix((np.concatenate(kv), (r, c)), shape=(nv, nv))
    return Mm, Km


def injection(prob: HDGProblem, n_vertices: int) -> sp.csr_matrix:
    """pi: P1 vertex values -> trace nodal values (linear along each facet)."""
    p = prob.prm.p
    rows, cols, vals = [], [], []
    for e in range(prob.n_facets):
        lo, hi = prob.facet_verts[e]
        for j in range(p + 1):
            t = j / p
            rows += [e * (p + 1) + j] * 2
            cols += [lo, hi]
            vals += [1.0 - t, t]
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.n_trace, n_vertices))


def nested_prolongation(parent: np.ndarray, n_coarse: int) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for i, (a, b) in enumerate(parent):
        if a == b:
            rows.append(i); cols.append(a); vals.append(1.0)
        else:
            rows += [i, i]; cols += [a, b]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(parent.shape[0], n_coarse))


class P1Multigrid:
    """Geometric V-cycle for the coarse problem on the nested P1 levels."""

    def __init__(self, ops: list, prolongs: list, nu1: int = 2, nu2: int = 2, omega: float = 2.0 / 3.0):
        self.ops = ops                   # finest first
        self.P = prolongs                # P[l]: level l+1 -> level l
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.dinv = [1.0 / A.diagonal() for A in ops]
        self.coarse_lu = spla.splu(ops[-1].tocsc())

    def vcycle(self, b: np.ndarray, lev: int = 0) -> np.ndarray:
        A = self.ops[lev]
        if lev == len(self.ops) - 1:
            return self.coarse_lu.solve(b)
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = x + self.omega * self.dinv[lev] * (b - A @ x)
        r = b - A @ x
        ec = self.vcycle(self.P[lev].T @ r, lev + 1)
        x = x + self.P[lev] @ ec
        for _ in range(self.nu2):
            x = x + self.omega * self.dinv[lev] * (b - A @ x)
        return x


# ------------------------------------------------------------------ Chebyshev smoother
#
# The paper smooths with a Chebyshev iteration (Sec. 5.2.1 and the solver
# configuration in the appendix: two Chebyshev steps, block-Jacobi/SOR
# preconditioned).  Here it is the Chebyshev iteration for D^-1 S (D the
# facet diagonal blocks) on an ellipse in the complex plane, centre theta on
# the real axis and focal half-distance delta (delta^2 < 0 when the ellipse
# is taller than wide, as under strong rotation).  With s_0 = 1/theta and
# s_k = 1 / (2 theta - delta^2 s_{k-1}),
#     x_1 = x_0 + s_0 D^-1 r_0,
#     x_{k+1} = x_k + 2 s_k D^-1 r_k + delta^2 s_k s_{k-1} (x_k - x_{k-1}),
# the error after n steps is T_n((theta - D^-1 S)/delta) / T_n(theta/delta)
# applied to the initial error; only delta^2 enters, so everything stays real.
# The ellipse is fitted to Ritz values of a few Arnoldi steps on D^-1 S:
# real extent [lower b, b] with b = grow * max Re(ritz) (PETSc's default
# Chebyshev bounds are 0.1 and 1.1 times the largest estimate), imaginary
# semi-axis grown until it holds every Ritz value with Re >= lower b.

def chebyshev_start_vector(n: int) -> np.ndarray:
    """Deterministic Arnoldi start vector: v_i = 1 + ((37 i) mod 101) / 101 for
    trace dof i in the lambda layout (facet-major, p+1 nodes per facet)."""
    i = np.arange(n, dtype=np.int64)
    return 1.0 + ((37 * i) % 101) / 101.0


def arnoldi_ritz(apply_op, v0: np.ndarray, k: int) -> np.ndarray:
    """Ritz values of k Arnoldi steps (modified Gram-Schmidt) from v0: the
    eigenvalues of the leading k x k block of the Hessenberg matrix."""
    n = v0.shape[0]
    k = min(k, n)
    V = np.zeros((k + 1, n))
    Hm = np.zeros((k + 1, k))
    V[0] = v0 / np.linalg.norm(v0)
    m = k
    for j in range(k):
        w = apply_op(V[j])
        for i in range(j + 1):
            Hm[i, j] = w @ V[i]
            w = w - Hm[i, j] * V[i]
        Hm[j + 1, j] = np.linalg.norm(w)
        if Hm[j + 1, j] <= 1e-14 * np.abs(Hm[:j + 1, j]).max():
            m = j + 1                      # invariant subspace: the Ritz values are exact
            break
        V[j + 1] = w / Hm[j + 1, j]
    return np.linalg.eigvals(Hm[:m, :m])


def chebyshev_ellipse(ritz: np.ndarray, lower: float = 0.1, grow: float = 1.1):
    """(theta, delta^2) of the ellipse fitted to the Ritz values (see above)."""
    b = grow * float(np.max(ritz.real))
    a = lower * b
    d, A = 0.5 * (a + b), 0.5 * (b - a)
    B2 = 0.0
    for z in ritz:
        if z.real >= a:
            q = 1.0 - ((z.real - d) / A) ** 2
            if q > 1e-3:
                B2 = max(B2, z.imag ** 2 / q)
    B2 *= grow * grow
    return d, A * A - B2


def chebyshev_polynomial(mu, theta: float, delta2: float, n: int):
    """Error-reduction factor T_n((theta - mu)/delta) / T_n(theta/delta) of n
    Chebyshev steps at the eigenvalue(s) mu of D^-1 S (closed form, complex)."""
    dl = np.sqrt(complex(delta2))
    if dl == 0:
        return (1.0 - np.asarray(mu, dtype=complex) / theta) ** n

    def T(z):
        t0, t1 = np.ones_like(z), z
        if n == 0:
            return t0
        for _ in range(n - 1):
            t0, t1 = t1, 2 * z * t1 - t0
        return t1

    mu = np.asarray(mu, dtype=complex)
    return T((theta - mu) / dl) / T(np.full_like(mu, theta / dl))


class TwoLevelPreconditioner:
    def __init__(self, prob: HDGProblem, mesh, S: sp.csr_matrix, n_pre: int = 2, n_post: int = 2,
                 omega: float = 2.0 / 3.0, coarse: str = "gmg", coarse_mode: str = "rotating",
                 p1_nu: tuple = (2, 2), p1_omega: float = 2.0 / 3.0, smoother: str = "jacobi",
                 cheb: tuple | None = None, cheb_steps: int = 20):
        self.prob, self.S = prob, S
        self.n_pre, self.n_post, self.omega = n_pre, n_post, omega
        self.smoother = smoother
        pp = prob.prm.p + 1
        # facet diagonal blocks D_e (rows and columns e(p+1) .. e(p+1)+p of S)
        # and their inverses, block-diagonal
        Sd = S.tocsr()
        nf = prob.n_facets
        idx = np.arange(nf)[:, None] * pp + np.arange(pp)[None, :]
        D = np.asarray(Sd[np.repeat(idx, pp, axis=1).ravel(), np.tile(idx, (1, pp)).ravel()]).reshape(nf, pp, pp)
        self.Dinv = sp.bsr_matrix((np.linalg.inv(D), np.arange(nf), np.arange(nf + 1)), shape=S.shape).tocsr()
        if smoother == "chebyshev":
            if cheb is None:
                ritz = arnoldi_ritz(lambda v: self.Dinv @ (S @ v), chebyshev_start_vector(S.shape[0]), cheb_steps)
                cheb = chebyshev_ellipse(ritz)
            self.cheb = (float(cheb[0]), float(cheb[1]))
        elif smoother != "jacobi":
            raise ValueError(smoother)
        nv = mesh.n_vertices
        self.Pi = injection(prob, nv)
        tau, g, H = prob.prm.tau, prob.prm.g, prob.prm.H
        levels = [mesh] + list(mesh.levels)
        if coarse_mode == "rotating":
            # f on the coarse levels by injection through the parent maps
            ops = []
            fv = prob.f_vertex
            for li, lev in enumerate(levels):
                if li > 0:
                    fv = coarse_vertex_values(fv, lev.parent, lev.n_vertices)
                ops.append(p1_rotating_operator(MeshData.of(lev), fv, tau, g, H).tocsr())
        elif coarse_mode == "rediscretised":
            ops = []
            for lev in levels:
                Mm, Km = p1_matrices(MeshData.of(lev))
                ops.append(((Mm + tau * tau * g * H * Km) / tau).tocsr())
        elif coarse_mode == "galerkin":
            ops = [(self.Pi.T @ S @ self.Pi).tocsr()]
        else:
            raise ValueError(coarse_mode)
        prolongs = [nested_prolongation(levels[l + 1].parent, levels[l + 1].n_vertices)
                    for l in range(len(levels) - 1)]
        if coarse_mode == "galerkin":
            for P in prolongs:
                ops.append((P.T @ ops[-1] @ P).tocsr())
        self.Sc = ops[0]
        if coarse == "exact" or len(ops) == 1:
            lu = spla.splu(ops[0].tocsc())
            self.coarse_solve = lu.solve
        elif coarse == "gmg":
            self.mg = P1Multigrid(ops, prolongs, p1_nu[0], p1_nu[1], p1_omega)
            self.coarse_solve = self.mg.vcycle
        elif coarse == "none":
            self.coarse_solve = lambda r: np.zeros_like(r)
        else:
            raise ValueError(coarse)

    def smooth(self, b: np.ndarray, x: np.ndarray, n: int) -> np.ndarray:
        if self.smoother == "jacobi":
            for _ in range(n):
                x = x + self.omega * (self.Dinv @ (b - self.S @ x))
            return x
        if n == 0:
            return x
        theta, delta2 = self.cheb
        s_prev = 1.0 / theta
        d = s_prev * (self.Dinv @ (b - self.S @ x))
        x = x + d
        for _ in range(1, n):
            s = 1.0 / (2.0 * theta - delta2 * s_prev)
            d = delta2 * s * s_prev * d + 2.0 * s * (self.Dinv @ (b - self.S @ x))
            x = x + d
            s_prev = s
        return x

    def __call__(self, b: np.ndarray) -> np.ndarray:
        x = self.smooth(b, np.zeros_like(b), self.n_pre)
        r = b - self.S @ x
        ec = self.coarse_solve(self.Pi.T @ r)
        x = x + self.Pi @ ec
        return self.smooth(b, x, self.n_post)


def solve_iterative(prob: HDGProblem, mesh, r_u, r_h, rtol: float = 1e-8, restart: int = 30,
                    maxiter: int = 500, **pc_kw):
    """Full oracle solve: step 1, FGMRES + V-cycle on the trace system, step 3."""
    S = prob.trace_operator()
    gvec = prob.condensed_rhs(r_u, r_h)
    pc = TwoLevelPreconditioner(prob, mesh, S, **pc_kw)
    lam, info = gmres(lambda v: S @ v, gvec, pc, restart=restart, rtol=rtol, maxiter=maxiter)
    u, h = prob.recover(lam, r_u, r_h)
    return (u, h), lam, info
