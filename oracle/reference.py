"""Reference-element data for the oracle, computed in exact rational arithmetic.

Test infrastructure only (see the package docstring).

* Cell space: P^p on the reference triangle (0,0), (1,0), (0,1)
  (Eq. DG_space_def), Lagrange basis at the equispaced nodes ``(a/p, b/p)``
  ordered row by row (``b`` outer, ``a`` inner).
* Trace space: P^p on a facet (Eq. DG_trace_def), Lagrange basis at
  ``t_j = j/p`` on ``[0, 1]``.
* Local edge ``i`` is the edge opposite vertex ``i``, traversed from vertex
  ``(i+1) % 3`` to vertex ``(i+2) % 3`` (counter-clockwise).

Polynomials are 2-D arrays of ``fractions.Fraction`` coefficients ``c[i, j]``
of ``xi^i eta^j``.  The Lagrange coefficients come from an exact Gauss-Jordan
inverse of the Vandermonde matrix and every integral is exact:
``int_T xi^i eta^j = i! j! / (i + j + 2)!`` on the triangle and
``int_0^1 t^k = 1/(k+1)`` on an edge.  Only the final matrices are rounded to
float64, so each entry is the correctly rounded exact value.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial

import numpy as np

REF_VERTS = ((Fraction(0), Fraction(0)), (Fraction(1), Fraction(0)), (Fraction(0), Fraction(1)))


def n_cell_nodes(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def cell_nodes_exact(p: int):
    return [(Fraction(a, p), Fraction(b, p)) for b in range(p + 1) for a in range(p + 1 - b)]


def cell_nodes(p: int) -> np.ndarray:
    return np.array([(float(x), float(y)) for (x, y) in cell_nodes_exact(p)])


def monomials(p: int):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


# ---------------------------------------------------------------- exact linear algebra

def exact_inverse(A):
    n = len(A)
    M = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                fac = M[r][c]
                M[r] = [a - fac * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


# ---------------------------------------------------------------- polynomials

def zeros2(a: int, b: int):
    return np.array([[Fraction(0)] * b for _ in range(a)], dtype=object)


def pmul(a, b):
    out = zeros2(a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1)
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0:
                for k in range(b.shape[0]):
                    for l in range(b.shape[1]):
                        if b[k, l] != 0:
                            out[i + k, j + l] += a[i, j] * b[k, l]
    return out


def dxi(a):
    out = zeros2(*a.shape)
    for i in range(1, a.shape[0]):
        for j in range(a.shape[1]):
            out[i - 1, j] = a[i, j] * i
    return out


def deta(a):
    out = zeros2(*a.shape)
    for i in range(a.shape[0]):
        for j in range(1, a.shape[1]):
            out[i, j - 1] = a[i, j] * j
    return out


def integrate_triangle(a) -> Fraction:
    s = Fraction(0)
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0:
                s += a[i, j] * Fraction(factorial(i) * factorial(j), factorial(i + j + 2))
    return s


def mul1(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pow1(a, k):
    out = [Fraction(1)]
    for _ in range(k):
        out = mul1(out, a)
    return out


def add1(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def on_segment(a, A, B):
    """1-D coefficients (in t) of ``a(A + t (B - A))``."""
    xi_t = [A[0], B[0] - A[0]]
    eta_t = [A[1], B[1] - A[1]]
    out = [Fraction(0)]
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0:
                term = [a[i, j] * c for c in mul1(pow1(xi_t, i), pow1(eta_t, j))]
                out = add1(out, term)
    return out


def integrate_unit(c) -> Fraction:
    return sum((ck / (k + 1) for k, ck in enumerate(c)), Fraction(0))


# ---------------------------------------------------------------- bases

@lru_cache(maxsize=None)
def cell_basis(p: int) -> tuple:
    """Lagrange basis of P^p as a tuple of 2-D Fraction coefficient arrays."""
    mons = monomials(p)
    nodes = cell_nodes_exact(p)
    V = [[x ** i * y ** j for (i, j) in mons] for (x, y) in nodes]
    C = exact_inverse(V)      # column n = coefficients of basis function n
    basis = []
    for n in range(len(nodes)):
        c = zeros2(p + 1, p + 1)
        for m, (i, j) in enumerate(mons):
            c[i, j] = C[m][n]
        basis.append(c)
    return tuple(basis)


@lru_cache(maxsize=None)
def trace_basis(p: int) -> tuple:
    """1-D Lagrange basis at t_j = j/p as Fraction coefficient lists in t."""
    t = [Fraction(j, p) for j in range(p + 1)]
    V = [[tj ** k for k in range(p + 1)] for tj in t]
    C = exact_inverse(V)
    return tuple([C[k][n] for k in range(p + 1)] for n in range(p + 1))


def barycentric() -> tuple:
    L0 = np.array([[Fraction(1), Fraction(-1)], [Fraction(-1), Fraction(0)]], dtype=object)
    L1 = np.array([[Fraction(0), Fraction(0)], [Fraction(1), Fraction(0)]], dtype=object)
    L2 = np.array([[Fraction(0), Fraction(1)], [Fraction(0), Fraction(0)]], dtype=object)
    return (L0, L1, L2)


def edge_endpoints(i: int):
    return REF_VERTS[(i + 1) % 3], REF_VERTS[(i + 2) % 3]


def _f(x) -> np.ndarray:
    return np.array(x, dtype=np.float64)


# ---------------------------------------------------------------- matrices

@lru_cache(maxsize=None)
def reference_matrices(p: int) -> dict:
    """Exact reference matrices, rounded once to float64.

    ``M[a,b] = int phi_a phi_b``; ``ML[i][a,b] = int L_i phi_a phi_b``;
    ``Dxi[a,b] = int phi_a d_xi phi_b`` (likewise ``Deta``);
    ``E[i][a,b] = int_0^1 phi_a phi_b`` along local edge i;
    ``N[i][a,j] = int_0^1 phi_a mu_j`` along local edge i;
    ``M1[j,k] = int_0^1 mu_j mu_k``.
    """
    phi = cell_basis(p)
    mu = trace_basis(p)
    L = barycentric()
    n = len(phi)
    M = [[integrate_triangle(pmul(phi[a], phi[b])) for b in range(n)] for a in range(n)]
    ML = [[[integrate_triangle(pmul(L[i], pmul(phi[a], phi[b]))) for b in range(n)]
           for a in range(n)] for i in range(3)]
    Dxi = [[integrate_triangle(pmul(phi[a], dxi(phi[b]))) for b in range(n)] for a in range(n)]
    Deta = [[integrate_triangle(pmul(phi[a], deta(phi[b]))) for b in range(n)] for a in range(n)]
    E, N = [], []
    for i in range(3):
        A, B = edge_endpoints(i)
        tr = [on_segment(phi[a], A, B) for a in range(n)]
        E.append(_f([[integrate_unit(mul1(tr[a], tr[b])) for b in range(n)] for a in range(n)]))
        N.append(_f([[integrate_unit(mul1(tr[a], mu[j])) for j in range(p + 1)] for a in range(n)]))
    M1 = [[integrate_unit(mul1(mu[j], mu[k])) for k in range(p + 1)] for j in range(p + 1)]
    return dict(M=_f(M), ML=[_f(x) for x in ML], Dxi=_f(Dxi), Deta=_f(Deta), E=E, N=N,
                M1=_f(M1), n=n)


def eval_cell_basis(p: int, xi: np.ndarray, eta: np.ndarray) -> np.ndarray:
    """Values of every basis function at points (xi, eta): ``[n_points, n_basis]``."""
    out = []
    for c in cell_basis(p):
        v = np.zeros_like(xi, dtype=np.float64)
        for i in range(c.shape[0]):
            for j in range(c.shape[1]):
                if c[i, j] != 0:
                    v = v + float(c[i, j]) * xi ** i * eta ** j
        out.append(v)
    return np.stack(out, axis=-1)
