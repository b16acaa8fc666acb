"""IMEX time stepping around the implicit solve (oracle; test infrastructure only).

The semi-discrete linear system is M dq/dt = N(q) + L(q) (Sec. 3, "Time
discretisation"): the fast gravity-wave terms L are treated implicitly, the
slower terms N explicitly.  For the linear equations N is the Coriolis term,
explicit as in the paper; the implicit operator of every stage is therefore the
upwind HDG operator with f = 0 and tau = alpha * dt (Eq. general_linear_system).

Operators.  The standard upwind DG matrix (oracle.stddg, equal to the HDG
system after eliminating the trace) is affine in tau: A(tau) = M + tau K, where
K holds the gravity-wave, stabilisation and (with f) Coriolis terms.  Two
assemblies give M = 2 A(1) - A(2) and K = A(2) - A(1); with f = 0 that is
K0 = -L, and K_f - K0 = C is the Coriolis part, N(q) = -C q.

Schemes.
* theta (Eq. theta_method): (M + theta dt K0) q1 = M q0 - dt (C q0 + (1 - theta) K0 q0).
* ARS2(2,3,2) (Eqs. IMEX_HDG_I, IMEX_HDG_II and the tableau of Sec.
  "Timestepping methods"): explicit a = [[0,0,0],[g,0,0],[d,1-d,0]],
  implicit a~ = [[0,0,0],[0,g,0],[0,1-g,g]], b = b~ = (0, 1-g, g), with
  g = 1 - 1/sqrt(2), d = -2 sqrt(2)/3.  Stage 1 is q0; stages 2 and 3 each
  solve (M + g dt K0) Q = rhs; the new state needs one more mass solve.

Each implicit stage is solved either directly (sparse LU of M + alpha dt K0)
or by the HDG route of the library (condense, solve for the trace, recover)
with r = M^-1 rhs; the two agree, which pins the operator extraction.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hdg import HDGProblem
from .stddg import assemble_standard_dg


class IMEXOperators:
    """M, K0 (gravity waves + upwind stabilisation, f = 0) and C (Coriolis)
    of the standard upwind DG system on one mesh; vectors are ordered as in
    oracle.stddg: cell, then component (u_x, u_y, h), then node."""

    def __init__(self, mesh, p: int, g: float, H: float, f_vertex: np.ndarray, tau_s: float | None = None):
        self.mesh, self.p, self.g, self.H, self.tau_s = mesh, p, g, H, tau_s
        self.f_zero = np.zeros_like(np.asarray(f_vertex, np.float64))
        probe = HDGProblem(mesh, p, 1.0, g, H, self.f_zero, tau_s=tau_s, lazy=True)
        self.N, self.np = probe.N, probe.np

        def pair(f):
            a1 = assemble_standard_dg(HDGProblem(mesh, p, 1.0, g, H, f, tau_s=tau_s))
            a2 = assemble_standard_dg(HDGProblem(mesh, p, 2.0, g, H, f, tau_s=tau_s))
            return a1, a2

        a1, a2 = pair(self.f_zero)
        self.M = (2.0 * a1 - a2).tocsc()
        self.K0 = (a2 - a1).tocsr()
        b1, b2 = pair(np.asarray(f_vertex, np.float64))
        self.C = ((b2 - b1) - self.K0).tocsr()
        self._mass = spla.splu(self.M)
        self._lu: dict[float, object] = {}
        self._hdg: dict[float, HDGProblem] = {}

    def mass(self, q: np.ndarray) -> np.ndarray:
        return self.M @ q

    def mass_solve(self, rhs: np.ndarray) -> np.ndarray:
        return self._mass.solve(rhs)

    def stage_solve(self, alpha_dt: float, rhs: np.ndarray, route: str = "direct") -> np.ndarray:
        """x with (M + alpha_dt K0) x = rhs: directly (sparse LU), or by the
        HDG route (tau = alpha_dt, f = 0, right-hand side function M^-1 rhs)."""
        if route == "direct":
            if alpha_dt not in self._lu:
                self._lu[alpha_dt] = spla.splu((self.M + alpha_dt * self.K0).tocsc())
            return self._lu[alpha_dt].solve(rhs)
        if alpha_dt not in self._hdg:
            self._hdg[alpha_dt] = HDGProblem(self.mesh, self.p, alpha_dt, self.g, self.H, self.f_zero,
                                             tau_s=self.tau_s)
        prob = self._hdg[alpha_dt]
        r = self.mass_solve(rhs).reshape(self.N, 3, self.np)
        (u, h), _ = prob.solve_condensed(r[:, :2, :], r[:, 2, :])
        return np.concatenate([u, h[:, None, :]], axis=1).ravel()

    def split(self, q: np.ndarray):
        qq = q.reshape(self.N, 3, self.np)
        return qq[:, :2, :], qq[:, 2, :]

    def energy(self, q: np.ndarray) -> float:
        """(H/g) ||u||^2 + ||h||^2 over the cells (L2, the mass matrix)."""
        qq, Mq = q.reshape(self.N, 3, self.np), self.mass(q).reshape(self.N, 3, self.np)
        return (self.H / self.g) * float(np.sum(qq[:, :2] * Mq[:, :2])) + float(np.sum(qq[:, 2] * Mq[:, 2]))

    def integral_of_h(self, q: np.ndarray) -> float:
        e = np.zeros((self.N, 3, self.np))
        e[:, 2, :] = 1.0
        return float(e.ravel() @ self.mass(q))


def theta_step(ops: IMEXOperators, q0: np.ndarray, dt: float, theta: float, route: str = "direct") -> np.ndarray:
    """One step of the theta method (Eq. theta_method), Coriolis explicit."""
    rhs = ops.mass(q0) - dt * (ops.C @ q0 + (1.0 - theta) * (ops.K0 @ q0))
    return ops.stage_solve(theta * dt, rhs, route)


ARS2_GAMMA = 1.0 - 1.0 / math.sqrt(2.0)
ARS2_DELTA = -2.0 * math.sqrt(2.0) / 3.0


def ars2_step(ops: IMEXOperators, q0: np.ndarray, dt: float, route: str = "direct") -> np.ndarray:
    """One step of ARS2(2,3,2) (Eqs. IMEX_HDG_I and IMEX_HDG_II)."""
    g, d = ARS2_GAMMA, ARS2_DELTA
    Mq0 = ops.mass(q0)
    Q1 = q0
    N1 = -(ops.C @ Q1)
    Q2 = ops.stage_solve(g * dt, Mq0 + dt * g * N1, route)
    N2, L2 = -(ops.C @ Q2), -(ops.K0 @ Q2)
    Q3 = ops.stage_solve(g * dt, Mq0 + dt * (d * N1 + (1.0 - d) * N2) + dt * (1.0 - g) * L2, route)
    N3, L3 = -(ops.C @ Q3), -(ops.K0 @ Q3)
    return ops.mass_solve(Mq0 + dt * ((1.0 - g) * (N2 + L2) + g * (N3 + L3)))


# Butcher tableaux (explicit a, implicit a~, weights b, b~) of the IMEX methods
# listed in the paper's section "Timestepping methods": ARS2(2,3,2),
# SSP2(3,2,2) and ARS3(4,4,3).
def _ars2():
    g, d = ARS2_GAMMA, ARS2_DELTA
    return ([[0, 0, 0], [g, 0, 0], [d, 1 - d, 0]], [[0, 0, 0], [0, g, 0], [0, 1 - g, g]],
            [0, 1 - g, g], [0, 1 - g, g])


TABLEAUX = {
    "ARS2": _ars2(),
    "SSP2": ([[0, 0, 0], [0, 0, 0], [0, 1, 0]], [[0.5, 0, 0], [-0.5, 0.5, 0], [0, 0.5, 0.5]],
             [0, 0.5, 0.5], [0, 0.5, 0.5]),
    "ARS3": ([[0, 0, 0, 0, 0], [1 / 2, 0, 0, 0, 0], [11 / 18, 1 / 18, 0, 0, 0], [5 / 6, -5 / 6, 1 / 2, 0, 0],
              [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0]],
             [[0, 0, 0, 0, 0], [0, 1 / 2, 0, 0, 0], [0, 1 / 6, 1 / 2, 0, 0], [0, -1 / 2, 1 / 2, 1 / 2, 0],
              [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2]],
             [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0], [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2]),
}


def imex_rk_step(ops: IMEXOperators, q0: np.ndarray, dt: float, tableau: str, route: str = "direct") -> np.ndarray:
    """One step of an s-stage IMEX method (Eqs. IMEX_HDG_I, IMEX_HDG_II):
    stage i solves M Q_i - a~_ii dt L(Q_i) = M q0 + dt sum_{j<i} (a_ij N(Q_j)
    + a~_ij L(Q_j)) (a plain mass solve where a~_ii = 0; stage 1 is q0 when
    nothing precedes it), then M q1 = M q0 + dt sum_i (b_i N(Q_i) + b~_i L(Q_i))."""
    a, at, b, bt = (np.asarray(x, dtype=float) for x in TABLEAUX[tableau])
    Mq0 = ops.mass(q0)
    Ns, Ls = [], []
    for i in range(len(b)):
        rhs = Mq0.copy()
        for j in range(i):
            rhs += dt * (a[i, j] * Ns[j] + at[i, j] * Ls[j])
        if at[i, i] != 0.0:
            Q = ops.stage_solve(at[i, i] * dt, rhs, route)
        elif i == 0:
            Q = q0
        else:
            Q = ops.mass_solve(rhs)
        Ns.append(-(ops.C @ Q))
        Ls.append(-(ops.K0 @ Q))
    upd = Mq0.copy()
    for i in range(len(b)):
        upd += dt * (b[i] * Ns[i] + bt[i] * Ls[i])
    return ops.mass_solve(upd)
