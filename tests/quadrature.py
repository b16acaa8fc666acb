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
