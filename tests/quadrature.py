"""Test helper: a collapsed (Duffy) Gauss-Legendre rule on the reference triangle.

Independent of the oracle's exact monomial integration; exact for polynomials
of degree <= 2n-2 in each collapsed variable, used to cross-check reference
matrices and to measure L2 errors against smooth exact solutions.
"""
import numpy as np


def triangle_rule(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    uu, vv = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    xi = uu.ravel()
    eta = (vv * (1.0 - uu)).ravel()
    wt = (wu * wv * (1.0 - uu)).ravel()
    return xi, eta, wt


def gauss_segment(n: int):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


class FloatLagrange:
    """Lagrange basis of P^p on the reference triangle at the equispaced nodes
    (a/p, b/p), b outer, built in floating point from a monomial Vandermonde
    solve: an independent construction (no exact rational arithmetic, no
    shared code) used to check the oracle's reference matrices entry by entry.
    """

    def __init__(self, p: int):
        self.p = p
        self.mons = [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]
        nodes = np.array([(a / p, b / p) for b in range(p + 1) for a in range(p + 1 - b)])
        V = np.array([[x ** i * y ** j for (i, j) in self.mons] for (x, y) in nodes])
        self.C = np.linalg.solve(V, np.eye(len(nodes)))      # column n: coefficients of phi_n

    def _mono(self, xi, eta, dx=0, dy=0):
        cols = []
        for (i, j) in self.mons:
            if i < dx or j < dy:
                cols.append(np.zeros_like(xi))
                continue
            ci = np.prod(np.arange(i, i - dx, -1)) if dx else 1.0
            cj = np.prod(np.arange(j, j - dy, -1)) if dy else 1.0
            cols.append(ci * cj * xi ** (i - dx) * eta ** (j - dy))
        return np.stack(cols, axis=-1)

    def values(self, xi, eta):
        return self._mono(xi, eta) @ self.C

    def d_xi(self, xi, eta):
        return self._mono(xi, eta, dx=1) @ self.C

    def d_eta(self, xi, eta):
        return self._mono(xi, eta, dy=1) @ self.C


def float_trace_basis(p: int, t):
    """1-D Lagrange basis at t_j = j/p on [0, 1] by the product formula."""
    nodes = np.arange(p + 1) / p
    out = np.ones((len(t), p + 1))
    for j in range(p + 1):
        for k in range(p + 1):
            if k != j:
                out[:, j] *= (t - nodes[k]) / (nodes[j] - nodes[k])
    return out
